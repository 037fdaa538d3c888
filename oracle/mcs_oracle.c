/*
 * mcs_oracle.c -- CPU oracle for the Monte Carlo DtN estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load it.  It shares no code with
 * the CUDA library: every formula below is written out again from the paper
 * and from the published methods it names.
 *
 * What it computes (Sec. 4.2 "Final Interior DtN Estimator", Alg. 2 and the
 * boxed interior estimator; Sec. 4.3 boxed exterior estimator, App. B.3-B.6):
 *   for every boundary row v: tangent ball (Sec. 5, bisection, 10 iterations;
 *   App. A item 3 radius clamp), W walks started on the ball surface with z
 *   importance-sampled by the ball jump kernel J^B(s,z) = 1/(2 pi |s-z|^3)
 *   (Eq. ball-jump-kernel) outside a cap of half-angle theta0 (Sec. 5),
 *   antithetic pairs (Sec. 5), walk-on-spheres to the eps-shell (Sec. 3
 *   "Walk-on-Spheres"), exit element -> column bin -> integer hit histogram.
 *   Exterior rows run the same in the Kelvin-inverted domain (Eq.
 *   exterior-jump-kernel-final, Eq. killing-measure-poisson-kernel).
 *
 * Closest point: brute force over ALL triangles, argmin by (d^2, triangle id).
 * Random numbers: Philox-4x32-10 (Salmon et al., SC'11) from its published
 * definition.  Floating point: compiled with -ffp-contract=off, so every
 * operation is one IEEE-754 round-to-nearest operation in the order written;
 * the CUDA path follows the same written operation order (the "arithmetic
 * contract" of the design notes), which is what makes hit counts comparable
 * bit for bit.  FP64 is the oracle's precision; the FP32 mode evaluates the
 * walk (start draw + steps + queries) in float and re-checks the eps-shell in
 * double, so that the FP32 kernel's integer decisions are taken in the
 * kernel's precision on both sides.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4 "Philox").        */
/* Ten rounds of two 32x32->64 multiplies with a bumped (Weyl) key.           */
/* ------------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* n counters (i_lo, i_hi, c2, c3) for i = start..start+n-1 -> 4n words */
void orc_philox_batch(uint64_t start, uint64_t n, uint32_t c2, uint32_t c3,
                      uint32_t k0, uint32_t k1, uint32_t *out)
{
    uint32_t key[2] = {k0, k1};
    for (uint64_t i = 0; i < n; i++) {
        uint64_t g = start + i;
        uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), c2, c3};
        orc_philox(ctr, key, out + 4 * i);
    }
}

/* uniforms on (0,1), symmetric, exactly representable */
static double uni64(uint32_t hi, uint32_t lo)
{
    uint64_t b = (((uint64_t)hi << 32) | (uint64_t)lo) >> 12;
    return (double)b * 0x1p-52 + 0x1p-53;
}
static float uni32(uint32_t x)
{
    return (float)(x >> 9) * 0x1p-23f + 0x1p-24f;
}

typedef struct { int f; double b[3]; } orc_exit;

#define TAG_RADIAL 0xFFFFFFFFu
#define KILL_KEY_XOR 0x4B494C4Cu
#define MAX_REJECT 32

/* ------------------------------------------------------------------------- */
/* problem description passed from Python                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    const double *V;  int nv;
    const int32_t *F; int nf;
    int n_rows;
    const double *row_pos;   /* n_rows x 3 */
    const double *row_nrm;   /* n_rows x 3 (unit, outward of Omega)          */
    const int32_t *tri2bin;  /* nf, or NULL: bin = argmax-barycentric vertex  */
    const int32_t *row_list; int n_list;   /* rows to simulate               */
    int walks;               /* W per row, even                              */
    double eps;
    int exterior;
    double origin[3];        /* exterior: inversion centre (inside Omega)    */
    uint64_t seed;
    double cap_deg;
    int bisect_iters;
    double kappa;
    int max_steps;
    double rho_min_factor;
    int prec;                /* 64 or 32 */
    int n_threads;
    long long killing_walks; /* exterior only; 0 = no killing walks           */
    int start_mode;          /* 0 importance-sampled ball (the estimator), 1  */
                             /* uniform on the ball outside the cap, weighted */
                             /* by q = A J^B / M; 2 naive inset (Alg. 1): one */
                             /* uniform WoS step from s - inset n, no cap     */
    double inset;            /* start_mode 2: inset distance h                */
    int walk_limit;          /* > 0: simulate only walks j < walk_limit of    */
                             /* each listed row (counters still use W); the   */
                             /* other exit records are -1                     */
} orc_problem;

typedef struct {
    int32_t *H;          /* n_list x n_rows hit counts                        */
    double  *Mjump;      /* n_list: importance-sampled ball jump mass M_v     */
    double  *kfac;       /* n_list: exterior |s~|^3 (1 for interior)          */
    int32_t *discarded;  /* n_list                                            */
    double  *r_t;        /* n_list: bisection radius                          */
    double  *rho;        /* n_list: empty-ball radius                         */
    double  *center;     /* n_list x 3: ball centre (inverted for exterior)   */
    int64_t *steps;      /* n_list: closest-point queries                     */
    int64_t *capped;     /* n_list                                            */
    int64_t *lost;       /* n_list: walks retired without a hit (exterior)    */
    int32_t *H0;         /* n_rows: killing-walk hits                         */
    int64_t *kill_stats; /* [steps, capped, lost]                             */
    int32_t *exit_tri;   /* optional n_list x W: exit triangle                */
    double  *exit_bary;  /* optional n_list x W x 3: exit barycentrics        */
    double  *walk_w;     /* optional n_list x W: the walk's weight q (1 in    */
                         /* modes 0 and 2)                                    */
} orc_result;

/* ------------------------------------------------------------------------- */
/* closest point on a triangle (Ericson, "Real-Time Collision Detection",    */
/* Sec. 5.1.5), written on (a, ab, ac); dot(x,y) = (x0*y0 + x1*y1) + x2*y2.   */
/* ------------------------------------------------------------------------- */
#define REAL double
#define SFX 64
#include "tri_impl.inc"
#undef REAL
#undef SFX
#define REAL float
#define SFX 32
#include "tri_impl.inc"
#undef REAL
#undef SFX

typedef struct {
    const orc_problem *pb;
    double *tri64;   /* nf x 9: a, ab, ac */
    float  *tri32;   /* nf x 9, from float-rounded vertices */
    double iw0;      /* 1 / sin(theta0/2) */
    double rmax;     /* tangent ball radius clamp */
    double rho0max;  /* exterior: radius of the empty ball at the inverted origin */
    double esc2;     /* exterior: |x~|^2 beyond which a walk has left the exterior's image */
    double cb[3];    /* interior: centre of the vertices' bounding box */
    double esc_int2; /* interior: squared box diagonal; a walk farther than this from cb has left the box */
} orc_ctx;

static void build_tris(orc_ctx *cx)
{
    const orc_problem *pb = cx->pb;
    cx->tri64 = (double *)malloc(sizeof(double) * 9 * (size_t)pb->nf);
    cx->tri32 = (float *)malloc(sizeof(float) * 9 * (size_t)pb->nf);
    for (int f = 0; f < pb->nf; f++) {
        const double *A = pb->V + 3 * pb->F[3 * f + 0];
        const double *B = pb->V + 3 * pb->F[3 * f + 1];
        const double *C = pb->V + 3 * pb->F[3 * f + 2];
        double *t = cx->tri64 + 9 * (size_t)f;
        float *s = cx->tri32 + 9 * (size_t)f;
        for (int i = 0; i < 3; i++) {
            t[i] = A[i];
            t[3 + i] = B[i] - A[i];
            t[6 + i] = C[i] - A[i];
            float a = (float)A[i], b = (float)B[i], c = (float)C[i];
            s[i] = a;
            s[3 + i] = b - a;
            s[6 + i] = c - a;
        }
    }
}

/* brute-force argmin over all triangles, lexicographic (d^2, id) */
static double closest_brute64(const orc_ctx *cx, const double p[3], int *fo, double bary[3])
{
    double best = INFINITY, bb[3] = {0, 0, 0};
    int bf = -1;
    for (int f = 0; f < cx->pb->nf; f++) {
        const double *t = cx->tri64 + 9 * (size_t)f;
        double b3[3];
        double d2 = tri_closest64(p, t, t + 3, t + 6, b3);
        if (d2 < best) { best = d2; bf = f; bb[0] = b3[0]; bb[1] = b3[1]; bb[2] = b3[2]; }
    }
    *fo = bf;
    bary[0] = bb[0]; bary[1] = bb[1]; bary[2] = bb[2];
    return best;
}
static float closest_brute32(const orc_ctx *cx, const float p[3], int *fo, float bary[3])
{
    float best = INFINITY, bb[3] = {0, 0, 0};
    int bf = -1;
    for (int f = 0; f < cx->pb->nf; f++) {
        const float *t = cx->tri32 + 9 * (size_t)f;
        float b3[3];
        float d2 = tri_closest32(p, t, t + 3, t + 6, b3);
        if (d2 < best) { best = d2; bf = f; bb[0] = b3[0]; bb[1] = b3[1]; bb[2] = b3[2]; }
    }
    *fo = bf;
    bary[0] = bb[0]; bary[1] = bb[1]; bary[2] = bb[2];
    return best;
}
static double dist64(const orc_ctx *cx, const double p[3])
{
    int f; double b[3];
    return sqrt(closest_brute64(cx, p, &f, b));
}

/* FP64 re-check of an FP32 exit against the float triangle f, widened exactly */
static double recheck64(const orc_ctx *cx, int f, const double p[3], double bary[3])
{
    const float *s = cx->tri32 + 9 * (size_t)f;
    double a[3], ab[3], ac[3];
    for (int i = 0; i < 3; i++) { a[i] = s[i]; ab[i] = s[3 + i]; ac[i] = s[6 + i]; }
    return tri_closest64(p, a, ab, ac, bary);
}

/* exit element -> column.  Vertex rows: the vertex of the exit triangle with
 * the largest barycentric weight (ties -> lower vertex index); sample rows:
 * the triangle's Voronoi owner (tri2bin). */
static int exit_bin(const orc_problem *pb, int f, const double bary[3])
{
    if (pb->tri2bin) return pb->tri2bin[f];
    int best = 0;
    for (int k = 1; k < 3; k++) {
        double bk = bary[k], bm = bary[best];
        int ik = pb->F[3 * f + k], im = pb->F[3 * f + best];
        if (bk > bm || (bk == bm && ik < im)) best = k;
    }
    return pb->F[3 * f + best];
}

/* ------------------------------------------------------------------------- */
/* samplers                                                                  */
/* ------------------------------------------------------------------------- */
/* uniform direction on S^2: Marsaglia (1972), rejection from the square */
static void dir64(uint32_t k0, uint32_t k1, uint32_t glo, uint32_t ghi, uint32_t step, double u[3])
{
    uint32_t key[2] = {k0, k1};
    for (uint32_t t = 0; t < MAX_REJECT; t++) {
        uint32_t ctr[4] = {glo, ghi, step, t}, x[4];
        orc_philox(ctr, key, x);
        double a = 2.0 * uni64(x[0], x[1]) - 1.0;
        double b = 2.0 * uni64(x[2], x[3]) - 1.0;
        double s = a * a + b * b;
        if (s < 1.0) {
            double h = sqrt(1.0 - s);
            u[0] = 2.0 * a * h;
            u[1] = 2.0 * b * h;
            u[2] = 1.0 - 2.0 * s;
            return;
        }
    }
    u[0] = 0.0; u[1] = 0.0; u[2] = 1.0;
}
static void dir32(uint32_t k0, uint32_t k1, uint32_t glo, uint32_t ghi, uint32_t step, float u[3])
{
    uint32_t key[2] = {k0, k1};
    for (uint32_t t = 0; t < MAX_REJECT; t++) {
        uint32_t ctr[4] = {glo, ghi, step, t}, x[4];
        orc_philox(ctr, key, x);
        float a = 2.0f * uni32(x[0]) - 1.0f;
        float b = 2.0f * uni32(x[2]) - 1.0f;
        float s = a * a + b * b;
        if (s < 1.0f) {
            float h = sqrtf(1.0f - s);
            u[0] = 2.0f * a * h;
            u[1] = 2.0f * b * h;
            u[2] = 1.0f - 2.0f * s;
            return;
        }
    }
    u[0] = 0.0f; u[1] = 0.0f; u[2] = 1.0f;
}

/* Orthonormal basis of a unit vector n: Duff, Burgess, Christensen, Hery,
 * Kensler, Liani, Villemin, "Building an Orthonormal Basis, Revisited",
 * JCGT 6(1), 2017 (its branchless formulas, restated). */
static void basis64(const double n[3], double e1[3], double e2[3])
{
    double sg = copysign(1.0, n[2]);
    double a = -1.0 / (sg + n[2]);
    double b = n[0] * n[1] * a;
    e1[0] = 1.0 + sg * n[0] * n[0] * a; e1[1] = sg * b; e1[2] = -(sg * n[0]);
    e2[0] = b; e2[1] = sg + n[1] * n[1] * a; e2[2] = -n[1];
}
static void basis32(const float n[3], float e1[3], float e2[3])
{
    float sg = copysignf(1.0f, n[2]);
    float a = -1.0f / (sg + n[2]);
    float b = n[0] * n[1] * a;
    e1[0] = 1.0f + sg * n[0] * n[0] * a; e1[1] = sg * b; e1[2] = -(sg * n[0]);
    e2[0] = b; e2[1] = sg + n[1] * n[1] * a; e2[2] = -n[1];
}

/* Start point of the pair (2q, 2q+1) on the empty ball B(c, rho) with pole
 * p = c + rho n.  The polar angle theta (from the pole, measured at c) is
 * drawn with density proportional to J^B(p, z) = 1/(2 pi |p-z|^3) on
 * theta > theta0: with w = sin(theta/2), |p - z| = 2 rho w and
 * dA = 4 rho^2 w dw dphi, so w has density ~ 1/w^2 on [w0, 1] and
 * 1/w = 1/w0 - u (1/w0 - 1).  The azimuth is uniform; the odd walk takes
 * phi + pi (antithetic pair, Sec. 5), which keeps |p - z|. */
/* Start points (Sec. 4.2).  mode 0: w = sin(theta/2) with pdf ~ 1/w^2 on
 * [w0, 1] (J^B importance sampling outside the cap theta < theta0); mode 1:
 * cos(theta) uniform on [-1, cos(theta0)] with the weight
 * q = |dB outside the cap| J^B(p, z) / M = (1 - w0^2) / (2 w^3 (1/w0 - 1));
 * mode 2: cos(theta) uniform on [-1, 1] (one WoS step, no cap), q = 1. */
static void start64(const orc_ctx *cx, uint32_t k0, uint32_t k1, uint64_t gp, int odd,
                    const double c[3], double rho, const double n[3], double z[3], int mode, double *q)
{
    uint32_t key[2] = {k0, k1}, x[4];
    uint32_t ctr[4] = {(uint32_t)gp, (uint32_t)(gp >> 32), 0u, TAG_RADIAL};
    orc_philox(ctr, key, x);
    double u = uni64(x[0], x[1]);
    double iw0 = cx->iw0;
    double w, cth;
    *q = 1.0;
    if (mode == 0) {
        double iw = iw0 - u * (iw0 - 1.0);
        w = 1.0 / iw;
        cth = 1.0 - 2.0 * (w * w);
    } else {
        double w0 = 1.0 / iw0;
        double c0 = mode == 1 ? 1.0 - 2.0 * (w0 * w0) : 1.0;
        cth = c0 - u * (c0 + 1.0);
        w = sqrt((1.0 - cth) * 0.5);
        if (mode == 1) *q = (1.0 - w0 * w0) / (2.0 * (w * w * w) * (iw0 - 1.0));
    }
    double sth = (2.0 * w) * sqrt(1.0 - w * w);
    double cph = 1.0, sph = 0.0;
    for (uint32_t t = 0; t < MAX_REJECT; t++) {
        uint32_t ct[4] = {(uint32_t)gp, (uint32_t)(gp >> 32), 0u, t};
        orc_philox(ct, key, x);
        double a = 2.0 * uni64(x[0], x[1]) - 1.0;
        double b = 2.0 * uni64(x[2], x[3]) - 1.0;
        double s = a * a + b * b;
        if (s < 1.0) { double r = sqrt(s); cph = a / r; sph = b / r; break; }
    }
    if (odd) { cph = -cph; sph = -sph; }
    double e1[3], e2[3];
    basis64(n, e1, e2);
    for (int i = 0; i < 3; i++)
        z[i] = c[i] + rho * (cth * n[i] + sth * (cph * e1[i] + sph * e2[i]));
}
static void start32(const orc_ctx *cx, uint32_t k0, uint32_t k1, uint64_t gp, int odd,
                    const float c[3], float rho, const float n[3], float z[3], int mode, double *q)
{
    uint32_t key[2] = {k0, k1}, x[4];
    uint32_t ctr[4] = {(uint32_t)gp, (uint32_t)(gp >> 32), 0u, TAG_RADIAL};
    orc_philox(ctr, key, x);
    float u = uni32(x[0]);
    float iw0 = (float)cx->iw0;
    float w, cth;
    *q = 1.0;
    if (mode == 0) {
        float iw = iw0 - u * (iw0 - 1.0f);
        w = 1.0f / iw;
        cth = 1.0f - 2.0f * (w * w);
    } else {
        float w0 = 1.0f / iw0;
        float c0 = mode == 1 ? 1.0f - 2.0f * (w0 * w0) : 1.0f;
        cth = c0 - u * (c0 + 1.0f);
        w = sqrtf((1.0f - cth) * 0.5f);
        if (mode == 1) {
            double wd = (double)w, w0d = 1.0 / cx->iw0;
            *q = (1.0 - w0d * w0d) / (2.0 * (wd * wd * wd) * (cx->iw0 - 1.0));
        }
    }
    float sth = (2.0f * w) * sqrtf(1.0f - w * w);
    float cph = 1.0f, sph = 0.0f;
    for (uint32_t t = 0; t < MAX_REJECT; t++) {
        uint32_t ct[4] = {(uint32_t)gp, (uint32_t)(gp >> 32), 0u, t};
        orc_philox(ct, key, x);
        float a = 2.0f * uni32(x[0]) - 1.0f;
        float b = 2.0f * uni32(x[2]) - 1.0f;
        float s = a * a + b * b;
        if (s < 1.0f) { float r = sqrtf(s); cph = a / r; sph = b / r; break; }
    }
    if (odd) { cph = -cph; sph = -sph; }
    float e1[3], e2[3];
    basis32(n, e1, e2);
    for (int i = 0; i < 3; i++)
        z[i] = c[i] + rho * (cth * n[i] + sth * (cph * e1[i] + sph * e2[i]));
}

/* ------------------------------------------------------------------------- */
/* walk-on-spheres (Sec. 3): jump to a uniform point of the largest empty     */
/* sphere until within eps; return the exit element.  A walk that reaches    */
/* max_steps queries exits at its current closest point and is counted.      */
/* ------------------------------------------------------------------------- */
static int walk_int64(const orc_ctx *cx, uint32_t k0, uint32_t k1, uint64_t g,
                      const double z[3], int64_t *steps, int *capped, int *lost, orc_exit *ex)
{
    const orc_problem *pb = cx->pb;
    double x[3] = {z[0], z[1], z[2]};
    for (int k = 1;; k++) {
        const double e0 = x[0] - cx->cb[0], e1 = x[1] - cx->cb[1], e2 = x[2] - cx->cb[2];
        if (e0 * e0 + e1 * e1 + e2 * e2 > cx->esc_int2) { *lost = 1; ex->f = -1; return -1; }  /* R18 */
        int f; double bary[3];
        double d = sqrt(closest_brute64(cx, x, &f, bary));
        (*steps)++;
        if (f < 0) { *capped = 1; ex->f = -1; return -1; }  /* non-finite point: lost */
        if (d < pb->eps || k == pb->max_steps) {
            *capped = !(d < pb->eps);
            ex->f = f; ex->b[0] = bary[0]; ex->b[1] = bary[1]; ex->b[2] = bary[2];
            return exit_bin(pb, f, bary);
        }
        double u[3];
        dir64(k0, k1, (uint32_t)g, (uint32_t)(g >> 32), (uint32_t)k, u);
        for (int i = 0; i < 3; i++) x[i] = x[i] + d * u[i];
    }
}
static int walk_int32(const orc_ctx *cx, uint32_t k0, uint32_t k1, uint64_t g,
                      const float z[3], int64_t *steps, int *capped, int *lost, orc_exit *ex)
{
    const orc_problem *pb = cx->pb;
    const float eps2 = (float)(2.0 * pb->eps);
    const float cb[3] = {(float)cx->cb[0], (float)cx->cb[1], (float)cx->cb[2]};
    const float esc = (float)cx->esc_int2;
    float x[3] = {z[0], z[1], z[2]};
    for (int k = 1;; k++) {
        const float e0 = x[0] - cb[0], e1 = x[1] - cb[1], e2 = x[2] - cb[2];
        if (e0 * e0 + e1 * e1 + e2 * e2 > esc) { *lost = 1; ex->f = -1; return -1; }  /* R18 */
        int f; float bary[3];
        float d = sqrtf(closest_brute32(cx, x, &f, bary));
        (*steps)++;
        if (f < 0) { *capped = 1; ex->f = -1; return -1; }
        if (d < eps2 || k == pb->max_steps) {
            double xd[3] = {x[0], x[1], x[2]}, b64[3];
            double d64 = sqrt(recheck64(cx, f, xd, b64));
            if (d64 < pb->eps || k == pb->max_steps) {
                *capped = !(d64 < pb->eps);
                ex->f = f; ex->b[0] = b64[0]; ex->b[1] = b64[1]; ex->b[2] = b64[2];
                return exit_bin(pb, f, b64);
            }
        }
        float u[3];
        dir32(k0, k1, (uint32_t)g, (uint32_t)(g >> 32), (uint32_t)k, u);
        for (int i = 0; i < 3; i++) x[i] = x[i] + d * u[i];
    }
}

/* Exterior walk in the Kelvin-inverted domain kappa(Omega^c) (Sec. 4.3).
 * At an inverted point x~ != 0 the primal point is x = x~/|x~|^2 (relative
 * to the inversion centre o).  The primal empty ball B(x, d) maps to an
 * inverted ball; the largest ball centred at x~ inside it has radius
 * d / (|x| (|x| + d)).  The ball B(0, 1/Rmax) is empty as well (all of the
 * surface lies within Rmax of o), so B(x~, 1/Rmax - |x~|) is a second valid
 * empty ball; the step uses the larger radius.  At x~ = 0 only the second
 * applies and no query is made; a walk that reaches the cap there is lost. */
static int walk_ext64(const orc_ctx *cx, uint32_t k0, uint32_t k1, uint64_t g,
                      const double z[3], int64_t *steps, int *capped, int *lost, orc_exit *ex)
{
    const orc_problem *pb = cx->pb;
    const double *o = pb->origin;
    double x[3] = {z[0], z[1], z[2]};
    for (int k = 1;; k++) {
        double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        double rho;
        if (r2 > cx->esc2) { *lost = 1; ex->f = -1; return -1; }  /* escaped (reading R17) */
        if (r2 == 0.0) {
            rho = cx->rho0max;
            if (k == pb->max_steps) { *capped = 1; *lost = 1; return -1; }
        } else {
            int f; double bary[3];
            double inv = 1.0 / r2;
            double xp[3], q[3];
            for (int i = 0; i < 3; i++) { xp[i] = x[i] * inv; q[i] = xp[i] + o[i]; }
            double d = sqrt(closest_brute64(cx, q, &f, bary));
            (*steps)++;
            if (f < 0) { *capped = 1; *lost = 1; ex->f = -1; return -1; }
            double nx = sqrt(xp[0] * xp[0] + xp[1] * xp[1] + xp[2] * xp[2]);
            double ri = d / (nx * (nx + d));
            double r0 = cx->rho0max - sqrt(r2);
            rho = ri > r0 ? ri : r0;
            if (rho < pb->eps || k == pb->max_steps) {
                *capped = !(rho < pb->eps);
                ex->f = f; ex->b[0] = bary[0]; ex->b[1] = bary[1]; ex->b[2] = bary[2];
                return exit_bin(pb, f, bary);
            }
        }
        double u[3];
        dir64(k0, k1, (uint32_t)g, (uint32_t)(g >> 32), (uint32_t)k, u);
        for (int i = 0; i < 3; i++) x[i] = x[i] + rho * u[i];
    }
}
static int walk_ext32(const orc_ctx *cx, uint32_t k0, uint32_t k1, uint64_t g,
                      const float z[3], int64_t *steps, int *capped, int *lost, orc_exit *ex)
{
    const orc_problem *pb = cx->pb;
    const float of[3] = {(float)pb->origin[0], (float)pb->origin[1], (float)pb->origin[2]};
    const float eps2 = (float)(2.0 * pb->eps);
    const float r0max = (float)cx->rho0max;
    const float esc2 = (float)cx->esc2;
    float x[3] = {z[0], z[1], z[2]};
    for (int k = 1;; k++) {
        float r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        float rho;
        if (r2 > esc2) { *lost = 1; ex->f = -1; return -1; }  /* escaped (reading R17) */
        if (r2 == 0.0f) {
            rho = r0max;
            if (k == pb->max_steps) { *capped = 1; *lost = 1; return -1; }
        } else {
            int f;
            float inv = 1.0f / r2;
            float xp[3], q[3], bary[3];
            for (int i = 0; i < 3; i++) { xp[i] = x[i] * inv; q[i] = xp[i] + of[i]; }
            float d = sqrtf(closest_brute32(cx, q, &f, bary));
            (*steps)++;
            if (f < 0) { *capped = 1; *lost = 1; ex->f = -1; return -1; }
            float nx = sqrtf(xp[0] * xp[0] + xp[1] * xp[1] + xp[2] * xp[2]);
            float ri = d / (nx * (nx + d));
            float r0 = r0max - sqrtf(r2);
            rho = ri > r0 ? ri : r0;
            if (rho < eps2 || k == pb->max_steps) {
                /* FP64 re-check of the eps-shell decision on triangle f */
                double b64[3];
                double xd[3] = {x[0], x[1], x[2]};
                double r2d = xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2];
                double invd = 1.0 / r2d;
                double xpd[3], qd[3];
                for (int i = 0; i < 3; i++) { xpd[i] = xd[i] * invd; qd[i] = xpd[i] + pb->origin[i]; }
                double dd = sqrt(recheck64(cx, f, qd, b64));
                double nxd = sqrt(xpd[0] * xpd[0] + xpd[1] * xpd[1] + xpd[2] * xpd[2]);
                double rid = dd / (nxd * (nxd + dd));
                double r0d = cx->rho0max - sqrt(r2d);
                double rhod = rid > r0d ? rid : r0d;
                if (rhod < pb->eps || k == pb->max_steps) {
                    *capped = !(rhod < pb->eps);
                    ex->f = f; ex->b[0] = b64[0]; ex->b[1] = b64[1]; ex->b[2] = b64[2];
                    return exit_bin(pb, f, b64);
                }
            }
        }
        float u[3];
        dir32(k0, k1, (uint32_t)g, (uint32_t)(g >> 32), (uint32_t)k, u);
        for (int i = 0; i < 3; i++) x[i] = x[i] + rho * u[i];
    }
}

/* ------------------------------------------------------------------------- */
/* tangent balls (Alg. 2 "LargestTangentBall"; Sec. 5: bisection, 10 its;     */
/* App. A item 3: radius clamp).  A radius r is accepted when the ball        */
/* centred at s - r n leaves a relative slack kappa: dist(c) >= (1-kappa) r.  */
/* The walk then uses the EMPTY ball centred at c with radius dist(c).        */
/* ------------------------------------------------------------------------- */
static void tangent_interior(const orc_ctx *cx, const double s[3], const double n[3],
                             double *r_out, double c[3], double *rho)
{
    const orc_problem *pb = cx->pb;
    const double onemk = 1.0 - pb->kappa;
    double rmax = cx->rmax, r;
    double cc[3];
    for (int i = 0; i < 3; i++) cc[i] = s[i] - rmax * n[i];
    if (dist64(cx, cc) >= onemk * rmax) {
        r = rmax;
    } else {
        double lo = 0.0, hi = rmax;
        for (int it = 0; it < pb->bisect_iters; it++) {
            double mid = 0.5 * (lo + hi);
            for (int i = 0; i < 3; i++) cc[i] = s[i] - mid * n[i];
            if (dist64(cx, cc) >= onemk * mid) lo = mid; else hi = mid;
        }
        r = lo;
    }
    for (int i = 0; i < 3; i++) c[i] = s[i] - r * n[i];
    *rho = dist64(cx, c);
    *r_out = r;
}

/* Exterior: rows are mapped to s~ = kappa(s - o); the inverted normal is the
 * Householder reflection of n about s^ with its sign flipped, -H n
 * (App. B.3, Eq. jacobian-times-normal).  The tangent ball lives in the
 * inverted domain (Sec. 4.3: the inverted jump kernel is an interior one and
 * takes the interior tangent-ball decomposition), so the slack is relative to
 * its inverted radius r, as for interior rows: the ball B(c~, (1-kappa) r),
 * c~ = s~ - r n~, must be empty.  An inverted ball B(c~, r') not containing 0
 * is the image of the primal ball with centre c~/(|c~|^2-r'^2) and radius
 * r'/(|c~|^2-r'^2), which one primal query tests.  (A slack taken on the
 * primal radius instead grows without bound as the inverted ball nears 0 and
 * lets the ball swallow other components.)  The accepted ball is replaced by
 * the image of the primal empty ball B(C, dist(C)) at the same primal centre,
 * which contains B(c~, (1-kappa) r). */
static int inv_ball_ok(const orc_ctx *cx, const double st[3], const double nt[3], double r,
                       double C[3], double *Rp)
{
    const orc_problem *pb = cx->pb;
    double ct[3];
    for (int i = 0; i < 3; i++) ct[i] = st[i] - r * nt[i];
    double cc = ct[0] * ct[0] + ct[1] * ct[1] + ct[2] * ct[2];
    double rk = (1.0 - pb->kappa) * r;
    double den = cc - rk * rk;
    /* the ball must stay clear of the inversion centre, and by a margin that
     * keeps its primal image ball (centre ~ 1/den) within FP64 resolution */
    if (!(den > 1e-6 * cc)) return 0;
    double inv = 1.0 / den, q[3];
    for (int i = 0; i < 3; i++) { C[i] = ct[i] * inv; q[i] = C[i] + pb->origin[i]; }
    *Rp = rk * inv;
    return dist64(cx, q) >= *Rp;
}

static void tangent_exterior(const orc_ctx *cx, const double s[3], const double n[3],
                             double *r_out, double c_inv[3], double *rho_inv,
                             double st[3], double nt[3], double *s3)
{
    const orc_problem *pb = cx->pb;
    double sp[3];
    for (int i = 0; i < 3; i++) sp[i] = s[i] - pb->origin[i];
    double r2s = sp[0] * sp[0] + sp[1] * sp[1] + sp[2] * sp[2];
    double inv = 1.0 / r2s;
    double sn = sp[0] * n[0] + sp[1] * n[1] + sp[2] * n[2];
    double t = (2.0 * sn) * inv;
    for (int i = 0; i < 3; i++) { st[i] = sp[i] * inv; nt[i] = sp[i] * t - n[i]; }
    *s3 = 1.0 / (r2s * sqrt(r2s));  /* |s~|^3 */
    double C[3], Rp, rmax = cx->rmax, r;
    if (inv_ball_ok(cx, st, nt, rmax, C, &Rp)) {
        r = rmax;
    } else {
        double lo = 0.0, hi = rmax;
        for (int it = 0; it < pb->bisect_iters; it++) {
            double mid = 0.5 * (lo + hi);
            if (inv_ball_ok(cx, st, nt, mid, C, &Rp)) lo = mid; else hi = mid;
        }
        r = lo;
    }
    *r_out = r;
    *rho_inv = 0.0;
    c_inv[0] = c_inv[1] = c_inv[2] = 0.0;
    if (!(r > 0.0)) return;
    /* recompute C for the accepted r (the last test may have been a rejection) */
    double ct[3];
    for (int i = 0; i < 3; i++) ct[i] = st[i] - r * nt[i];
    double cc = ct[0] * ct[0] + ct[1] * ct[1] + ct[2] * ct[2];
    double rk = (1.0 - pb->kappa) * r;
    double den = cc - rk * rk;
    if (!(den > 1e-6 * cc)) return;
    double invd = 1.0 / den, q[3];
    for (int i = 0; i < 3; i++) { C[i] = ct[i] * invd; q[i] = C[i] + pb->origin[i]; }
    double D = dist64(cx, q);
    double CC = C[0] * C[0] + C[1] * C[1] + C[2] * C[2];
    double den2 = CC - D * D;
    /* |C|^2 - D^2 cancels when the empty ball nearly reaches the centre */
    if (!(den2 > 1e-8 * CC)) return;
    double inv2 = 1.0 / den2;
    for (int i = 0; i < 3; i++) c_inv[i] = C[i] * inv2;
    *rho_inv = D * inv2;
}

/* ------------------------------------------------------------------------- */
/* AABB clamp (App. A item 3): maximum tangent-ball radius = half the        */
/* shortest side of the surface's axis-aligned bounding box (of the          */
/* Kelvin-inverted vertices for the exterior).                               */
/* ------------------------------------------------------------------------- */
static double rmax_of(const orc_problem *pb)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < pb->nv; v++) {
        double p[3];
        if (pb->exterior) {
            double d[3];
            for (int i = 0; i < 3; i++) d[i] = pb->V[3 * v + i] - pb->origin[i];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double inv = 1.0 / r2;
            for (int i = 0; i < 3; i++) p[i] = d[i] * inv;
        } else {
            for (int i = 0; i < 3; i++) p[i] = pb->V[3 * v + i];
        }
        for (int i = 0; i < 3; i++) {
            if (p[i] < lo[i]) lo[i] = p[i];
            if (p[i] > hi[i]) hi[i] = p[i];
        }
    }
    double m = hi[0] - lo[0];
    if (hi[1] - lo[1] < m) m = hi[1] - lo[1];
    if (hi[2] - lo[2] < m) m = hi[2] - lo[2];
    return 0.5 * m;
}

static double rho0max_of(const orc_problem *pb)
{
    double m = 0.0;
    for (int v = 0; v < pb->nv; v++) {
        double d[3];
        for (int i = 0; i < 3; i++) d[i] = pb->V[3 * v + i] - pb->origin[i];
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r > m) m = r;
    }
    return 1.0 / m;
}

/* Exterior walks live in the Kelvin image of the unbounded component of the
 * complement of the surface.  The inversion centre o lies in a bounded
 * component, and the ball B(o, dist(o)) holds no surface point, so it lies in
 * o's component too: no point of the exterior is closer to o than dist(o),
 * and the exterior's image satisfies |x~| <= 1/dist(o).  A walk found at
 * |x~| > 2/dist(o) is in o's own component (it started in a pocket of a
 * self-overlapping surface that contains o, or crossed the surface); it can
 * never reach the eps-shell of the exterior's boundary and would run off to
 * |x~| = infinity, so it is retired without a hit (reading R17). */
static double esc2_of(const orc_ctx *cx)
{
    const double d = dist64(cx, cx->pb->origin);
    return d > 0.0 ? 4.0 / (d * d) : INFINITY;
}

/* Interior walks live in bounded components of the complement of the
 * surface, all inside the bounding box of the vertices.  A walk farther from
 * the box centre than the box diagonal (twice the box's circumradius) is in
 * the unbounded component -- its row's inward side faces outward (a face
 * whose orientation repair failed) -- and could only come back by chance; it
 * is retired without a hit (reading R18). */
static void interior_bound(orc_ctx *cx)
{
    const orc_problem *pb = cx->pb;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < pb->nv; v++)
        for (int i = 0; i < 3; i++) {
            if (pb->V[3 * v + i] < lo[i]) lo[i] = pb->V[3 * v + i];
            if (pb->V[3 * v + i] > hi[i]) hi[i] = pb->V[3 * v + i];
        }
    for (int i = 0; i < 3; i++) cx->cb[i] = 0.5 * (lo[i] + hi[i]);
    const double s0 = hi[0] - lo[0], s1 = hi[1] - lo[1], s2 = hi[2] - lo[2];
    cx->esc_int2 = s0 * s0 + s1 * s1 + s2 * s2;
}

static void ctx_init(orc_ctx *cx, const orc_problem *pb)
{
    cx->pb = pb;
    interior_bound(cx);
    build_tris(cx);
    cx->iw0 = 1.0 / sin(pb->cap_deg * (M_PI / 360.0));
    cx->rmax = rmax_of(pb);
    cx->rho0max = pb->exterior ? rho0max_of(pb) : 0.0;
    cx->esc2 = pb->exterior ? esc2_of(cx) : INFINITY;
}
static void ctx_free(orc_ctx *cx)
{
    free(cx->tri64);
    free(cx->tri32);
}

/* ------------------------------------------------------------------------- */
/* the estimator: rows x walks -> hit histogram H, plus per-row weights      */
/* ------------------------------------------------------------------------- */
int orc_estimate(const orc_problem *pb, orc_result *res)
{
    orc_ctx cx;
    ctx_init(&cx, pb);
    const uint32_t k0 = (uint32_t)pb->seed, k1 = (uint32_t)(pb->seed >> 32);
    const double iw0 = cx.iw0;
#ifdef _OPENMP
    if (pb->n_threads > 0) omp_set_num_threads(pb->n_threads);
#endif
    #pragma omp parallel for schedule(dynamic, 1)
    for (int li = 0; li < pb->n_list; li++) {
        const int v = pb->row_list ? pb->row_list[li] : li;
        const double *s = pb->row_pos + 3 * v, *n = pb->row_nrm + 3 * v;
        int32_t *Hrow = res->H + (size_t)li * pb->n_rows;
        double r = 0.0, c[3] = {0, 0, 0}, rho = 0.0, nb[3] = {n[0], n[1], n[2]}, s3 = 1.0;
        int nz = (n[0] != 0.0 || n[1] != 0.0 || n[2] != 0.0);
        if (nz) {
            if (pb->exterior) {
                double st[3];
                tangent_exterior(&cx, s, n, &r, c, &rho, st, nb, &s3);
            } else if (pb->start_mode == 2) {
                /* naive estimator (Alg. 1): the walk starts at the inset point */
                for (int i = 0; i < 3; i++) c[i] = s[i] - pb->inset * n[i];
                r = pb->inset;
                rho = dist64(&cx, c);
            } else {
                tangent_interior(&cx, s, n, &r, c, &rho);
            }
        }
        res->r_t[li] = r;
        res->rho[li] = rho;
        res->center[3 * li + 0] = c[0];
        res->center[3 * li + 1] = c[1];
        res->center[3 * li + 2] = c[2];
        res->kfac[li] = s3;
        const int disc = !nz || !(rho >= pb->rho_min_factor * pb->eps);
        res->discarded[li] = disc;
        res->steps[li] = 0;
        res->capped[li] = 0;
        if (res->lost) res->lost[li] = 0;
        if (disc) {
            res->Mjump[li] = 0.0;
            if (res->exit_tri)
                for (int j = 0; j < pb->walks; j++) res->exit_tri[(size_t)li * pb->walks + j] = -1;
            continue;
        }
        /* importance-sampled jump mass over theta > theta0:
         * int J^B(p,z) dz = (1/w0 - 1) / (2 rho) */
        res->Mjump[li] = pb->start_mode == 2 ? 1.0 / pb->inset : (iw0 - 1.0) / (2.0 * rho);
        const float cf[3] = {(float)c[0], (float)c[1], (float)c[2]};
        const float nf3[3] = {(float)nb[0], (float)nb[1], (float)nb[2]};
        const float rf = (float)rho;
        const int nwalk = pb->walk_limit > 0 && pb->walk_limit < pb->walks ? pb->walk_limit : pb->walks;
        if (res->exit_tri)
            for (int j = nwalk; j < pb->walks; j++) res->exit_tri[(size_t)li * pb->walks + j] = -1;
        for (int j = 0; j < nwalk; j++) {
            uint64_t g = (uint64_t)v * (uint64_t)pb->walks + (uint64_t)j;
            uint64_t gp = g - (uint64_t)(j & 1);
            int capped = 0, lost = 0, bin;
            orc_exit ex = {-1, {0, 0, 0}};
            double q = 1.0;
            if (pb->prec == 32) {
                float z[3];
                start32(&cx, k0, k1, gp, j & 1, cf, rf, nf3, z, pb->start_mode, &q);
                bin = pb->exterior ? walk_ext32(&cx, k0, k1, g, z, &res->steps[li], &capped, &lost, &ex)
                                   : walk_int32(&cx, k0, k1, g, z, &res->steps[li], &capped, &lost, &ex);
            } else {
                double z[3];
                start64(&cx, k0, k1, gp, j & 1, c, rho, nb, z, pb->start_mode, &q);
                bin = pb->exterior ? walk_ext64(&cx, k0, k1, g, z, &res->steps[li], &capped, &lost, &ex)
                                   : walk_int64(&cx, k0, k1, g, z, &res->steps[li], &capped, &lost, &ex);
            }
            res->capped[li] += capped;
            if (res->lost) res->lost[li] += lost;
            if (bin >= 0) Hrow[bin] += 1;
            if (res->exit_tri) {
                size_t e = (size_t)li * pb->walks + j;
                res->exit_tri[e] = ex.f;
                res->exit_bary[3 * e] = ex.b[0];
                res->exit_bary[3 * e + 1] = ex.b[1];
                res->exit_bary[3 * e + 2] = ex.b[2];
            }
            if (res->walk_w) res->walk_w[(size_t)li * pb->walks + j] = q;
        }
    }
    /* killing walks from the inverted origin (Eq. killing-measure-poisson-kernel) */
    if (pb->exterior && pb->killing_walks > 0) {
        const uint32_t q0 = k0, q1 = k1 ^ KILL_KEY_XOR;
        int64_t st = 0, cp = 0, ls = 0;
        #pragma omp parallel for schedule(dynamic, 64) reduction(+ : st, cp, ls)
        for (long long i = 0; i < pb->killing_walks; i++) {
            int capped = 0, lost = 0, bin;
            int64_t s1 = 0;
            orc_exit ex;
            if (pb->prec == 32) {
                float z[3] = {0.0f, 0.0f, 0.0f};
                bin = walk_ext32(&cx, q0, q1, (uint64_t)i, z, &s1, &capped, &lost, &ex);
            } else {
                double z[3] = {0.0, 0.0, 0.0};
                bin = walk_ext64(&cx, q0, q1, (uint64_t)i, z, &s1, &capped, &lost, &ex);
            }
            st += s1; cp += capped; ls += lost;
            if (bin >= 0) {
                #pragma omp atomic
                res->H0[bin] += 1;
            }
        }
        res->kill_stats[0] = st; res->kill_stats[1] = cp; res->kill_stats[2] = ls;
    }
    ctx_free(&cx);
    return 0;
}

/* Walks started at given points (primal coordinates), W each: exit triangle
 * and barycentrics of every walk.  Walk j of point i uses g = i*W + j; the
 * exterior version starts at kappa(x - o).  Used by the harmonic-function
 * tests (Eq. poisson-kernel-probabilistic, Eq. poisson-kernel-kelvin). */
int orc_walk_from_points(const orc_problem *pb, const double *X, int npts,
                         int32_t *exit_tri, double *exit_bary, int64_t *steps_out, int64_t *capped_out)
{
    orc_ctx cx;
    ctx_init(&cx, pb);
    const uint32_t k0 = (uint32_t)pb->seed, k1 = (uint32_t)(pb->seed >> 32);
#ifdef _OPENMP
    if (pb->n_threads > 0) omp_set_num_threads(pb->n_threads);
#endif
    int64_t st = 0, cp = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(+ : st, cp)
    for (int i = 0; i < npts; i++) {
        for (int j = 0; j < pb->walks; j++) {
            uint64_t g = (uint64_t)i * (uint64_t)pb->walks + (uint64_t)j;
            int capped = 0, lost = 0;
            int64_t s1 = 0;
            orc_exit ex = {-1, {0, 0, 0}};
            double z[3];
            if (pb->exterior) {
                double d[3];
                for (int k = 0; k < 3; k++) d[k] = X[3 * i + k] - pb->origin[k];
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double inv = 1.0 / r2;
                for (int k = 0; k < 3; k++) z[k] = d[k] * inv;
            } else {
                for (int k = 0; k < 3; k++) z[k] = X[3 * i + k];
            }
            if (pb->prec == 32) {
                float zf[3] = {(float)z[0], (float)z[1], (float)z[2]};
                if (pb->exterior) walk_ext32(&cx, k0, k1, g, zf, &s1, &capped, &lost, &ex);
                else walk_int32(&cx, k0, k1, g, zf, &s1, &capped, &lost, &ex);
            } else {
                if (pb->exterior) walk_ext64(&cx, k0, k1, g, z, &s1, &capped, &lost, &ex);
                else walk_int64(&cx, k0, k1, g, z, &s1, &capped, &lost, &ex);
            }
            size_t e = (size_t)i * pb->walks + j;
            exit_tri[e] = ex.f;
            exit_bary[3 * e] = ex.b[0]; exit_bary[3 * e + 1] = ex.b[1]; exit_bary[3 * e + 2] = ex.b[2];
            st += s1; cp += capped;
        }
    }
    steps_out[0] = st; capped_out[0] = cp;
    ctx_free(&cx);
    return 0;
}

/* interior tangent balls of all rows (used to place the inversion centre) */
int orc_tangent_balls(const orc_problem *pb, double *r_out, double *c_out, double *rho_out)
{
    orc_problem p2 = *pb;
    p2.exterior = 0;
    orc_ctx cx;
    ctx_init(&cx, &p2);
#ifdef _OPENMP
    if (pb->n_threads > 0) omp_set_num_threads(pb->n_threads);
#endif
    #pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < pb->n_rows; v++) {
        const double *s = pb->row_pos + 3 * v, *n = pb->row_nrm + 3 * v;
        if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) {
            r_out[v] = 0.0; rho_out[v] = 0.0;
            c_out[3 * v] = s[0]; c_out[3 * v + 1] = s[1]; c_out[3 * v + 2] = s[2];
            continue;
        }
        tangent_interior(&cx, s, n, &r_out[v], c_out + 3 * v, &rho_out[v]);
    }
    ctx_free(&cx);
    return 0;
}

/* brute-force closest point of many query points (FP64 and FP32) */
void orc_closest_points(const double *V, int nv, const int32_t *F, int nf, const double *P, int np,
                        int prec, double *d2_out, int32_t *f_out, double *bary_out)
{
    orc_problem pb;
    memset(&pb, 0, sizeof pb);
    pb.V = V; pb.nv = nv; pb.F = F; pb.nf = nf;
    orc_ctx cx;
    cx.pb = &pb;
    build_tris(&cx);
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < np; i++) {
        int f;
        if (prec == 32) {
            float p[3] = {(float)P[3 * i], (float)P[3 * i + 1], (float)P[3 * i + 2]}, b[3];
            float d2 = closest_brute32(&cx, p, &f, b);
            d2_out[i] = d2;
            bary_out[3 * i] = b[0]; bary_out[3 * i + 1] = b[1]; bary_out[3 * i + 2] = b[2];
        } else {
            double b[3];
            d2_out[i] = closest_brute64(&cx, P + 3 * i, &f, b);
            bary_out[3 * i] = b[0]; bary_out[3 * i + 1] = b[1]; bary_out[3 * i + 2] = b[2];
        }
        f_out[i] = f;
    }
    free(cx.tri64);
    free(cx.tri32);
}

/* sampler probes for the distribution tests */
void orc_directions(uint64_t seed, uint64_t g, uint32_t nsteps, int prec, double *u_out)
{
    for (uint32_t k = 1; k <= nsteps; k++) {
        if (prec == 32) {
            float u[3];
            dir32((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)g, (uint32_t)(g >> 32), k, u);
            for (int i = 0; i < 3; i++) u_out[3 * (k - 1) + i] = u[i];
        } else {
            dir64((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)g, (uint32_t)(g >> 32), k, u_out + 3 * (k - 1));
        }
    }
}

void orc_start_points(uint64_t seed, double cap_deg, const double c[3], double rho, const double n[3],
                      uint64_t npairs, int prec, double *z_out)
{
    orc_problem pb;
    memset(&pb, 0, sizeof pb);
    orc_ctx cx;
    cx.pb = &pb;
    cx.iw0 = 1.0 / sin(cap_deg * (M_PI / 360.0));
    for (uint64_t q = 0; q < npairs; q++) {
        for (int odd = 0; odd < 2; odd++) {
            double *z = z_out + 3 * (2 * q + odd);
            if (prec == 32) {
                float cf[3] = {(float)c[0], (float)c[1], (float)c[2]};
                float nf3[3] = {(float)n[0], (float)n[1], (float)n[2]}, zf[3];
                double qw;
                start32(&cx, (uint32_t)seed, (uint32_t)(seed >> 32), 2 * q, odd, cf, (float)rho, nf3, zf, 0, &qw);
                z[0] = zf[0]; z[1] = zf[1]; z[2] = zf[2];
            } else {
                double qw;
                start64(&cx, (uint32_t)seed, (uint32_t)(seed >> 32), 2 * q, odd, c, rho, n, z, 0, &qw);
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* row setup                                                                 */
/* ------------------------------------------------------------------------- */
/* Vertex rows (lumped P1 basis): n_v = normalised sum of the (unnormalised)
 * face normals (b-a)x(c-a) of the faces containing v, in ascending face id;
 * A_v = (sum of incident face areas) / 3.  A vertex with a zero normal sum
 * gets n_v = 0 and is discarded by the estimator. */
void orc_vertex_rows(const double *V, int nv, const int32_t *F, int nf,
                     double *pos, double *nrm, double *area)
{
    double *S = (double *)calloc(3 * (size_t)nv, sizeof(double));
    double *A = (double *)calloc((size_t)nv, sizeof(double));
    for (int f = 0; f < nf; f++) {
        const double *a = V + 3 * F[3 * f], *b = V + 3 * F[3 * f + 1], *c = V + 3 * F[3 * f + 2];
        double ab[3], ac[3], N[3];
        for (int i = 0; i < 3; i++) { ab[i] = b[i] - a[i]; ac[i] = c[i] - a[i]; }
        N[0] = ab[1] * ac[2] - ab[2] * ac[1];
        N[1] = ab[2] * ac[0] - ab[0] * ac[2];
        N[2] = ab[0] * ac[1] - ab[1] * ac[0];
        double ar = 0.5 * sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        for (int k = 0; k < 3; k++) {
            int v = F[3 * f + k];
            S[3 * v] += N[0]; S[3 * v + 1] += N[1]; S[3 * v + 2] += N[2];
            A[v] += ar;
        }
    }
    for (int v = 0; v < nv; v++) {
        double *s = S + 3 * v;
        double l = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
        for (int i = 0; i < 3; i++) {
            pos[3 * v + i] = V[3 * v + i];
            nrm[3 * v + i] = l > 0.0 ? s[i] / l : 0.0;
        }
        area[v] = A[v] / 3.0;
    }
    free(S);
    free(A);
}

/* solid angle of triangle (a,b,c) seen from q: Van Oosterom & Strackee,
 * IEEE TBME 30(2), 1983: tan(Omega/2) = det[a b c] /
 * (|a||b||c| + (a.b)|c| + (b.c)|a| + (c.a)|b|), with a,b,c relative to q. */
static double solid_angle(const double *A, const double *B, const double *C, const double q[3])
{
    double a[3], b[3], c[3];
    for (int i = 0; i < 3; i++) { a[i] = A[i] - q[i]; b[i] = B[i] - q[i]; c[i] = C[i] - q[i]; }
    double la = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double lb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    double lc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                 a[2] * (b[0] * c[1] - b[1] * c[0]);
    double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    double bc = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
    double ca = c[0] * a[0] + c[1] * a[1] + c[2] * a[2];
    double den = la * lb * lc + ab * lc + bc * la + ca * lb;
    return 2.0 * atan2(det, den);
}

/* generalized winding number (Jacobson, Kavan, Sorkine-Hornung 2013):
 * sum of signed solid angles / 4 pi, optionally skipping one face */
double orc_gwn_skip(const double *V, const int32_t *F, int nf, const double q[3], int skip)
{
    double s = 0.0;
    for (int f = 0; f < nf; f++)
        if (f != skip) s += solid_angle(V + 3 * F[3 * f], V + 3 * F[3 * f + 1], V + 3 * F[3 * f + 2], q);
    return s / (4.0 * M_PI);
}
double orc_gwn(const double *V, const int32_t *F, int nf, const double q[3])
{
    return orc_gwn_skip(V, F, nf, q, -1);
}

/* Sample rows: farthest-point sampling over face centroids, starting at
 * face 0 (the point basis of Sec. 4.4, FPS standing in for blue noise).
 * Each face is owned by its nearest selected sample (first selected on a
 * tie); a sample's quadrature area is the total area of the faces it owns
 * and tri2bin maps each face to its owner.  The row normal is the unit face
 * normal of the sampled face, optionally oriented by the generalized
 * winding number (App. A item 1) of the OTHER faces, which rises towards
 * the inside across the face: keep n when GWN'(x - delta n) > GWN'(x +
 * delta n), delta = sqrt(area_f)/4, flip it otherwise. */
void orc_fps_rows(const double *V, int nv, const int32_t *F, int nf, int ns, int orient,
                  const int32_t *orient_list, int n_orient,
                  int32_t *sel, double *pos, double *nrm, double *area, int32_t *tri2bin)
{
    (void)nv;
    double *cen = (double *)malloc(sizeof(double) * 3 * (size_t)nf);
    float *cenf = (float *)malloc(sizeof(float) * 3 * (size_t)nf);
    float *mind = (float *)malloc(sizeof(float) * (size_t)nf);
    double *far_ = (double *)malloc(sizeof(double) * (size_t)nf);
    for (int f = 0; f < nf; f++) {
        const double *a = V + 3 * F[3 * f], *b = V + 3 * F[3 * f + 1], *c = V + 3 * F[3 * f + 2];
        for (int i = 0; i < 3; i++) cen[3 * f + i] = ((a[i] + b[i]) + c[i]) / 3.0;
        double ab[3], ac[3], N[3];
        for (int i = 0; i < 3; i++) { ab[i] = b[i] - a[i]; ac[i] = c[i] - a[i]; }
        N[0] = ab[1] * ac[2] - ab[2] * ac[1];
        N[1] = ab[2] * ac[0] - ab[0] * ac[2];
        N[2] = ab[0] * ac[1] - ab[1] * ac[0];
        far_[f] = 0.5 * sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        for (int i = 0; i < 3; i++) cenf[3 * f + i] = (float)cen[3 * f + i];
        mind[f] = INFINITY;
        tri2bin[f] = -1;
    }
    /* greedy farthest points in single precision on the float-rounded
     * centroids (reading R16): the squared distance is ((dx dx + dy dy) + dz dz)
     * in float; a face's owner is the first sample strictly nearest; the next
     * sample is the face with the largest distance, lowest face id on ties */
    /* the faces are split into contiguous ranges over the threads; each
     * range's first maximum, then the largest value, lowest face on ties:
     * the same choice as one ascending scan */
    sel[0] = 0;
    for (int i = 0; i < ns; i++) {
        const float *q = cenf + 3 * sel[i];
        int arg = 0;
        float best = -1.0f;
        #pragma omp parallel
        {
            int targ = 0;
            float tbest = -1.0f;
            #pragma omp for schedule(static)
            for (int f = 0; f < nf; f++) {
                float d[3] = {cenf[3 * f] - q[0], cenf[3 * f + 1] - q[1], cenf[3 * f + 2] - q[2]};
                float d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (d2 < mind[f]) { mind[f] = d2; tri2bin[f] = i; }
                if (mind[f] > tbest) { tbest = mind[f]; targ = f; }
            }
            #pragma omp critical
            {
                if (tbest > best || (tbest == best && targ < arg)) { best = tbest; arg = targ; }
            }
        }
        if (i + 1 < ns) sel[i + 1] = arg;
    }
    for (int i = 0; i < ns; i++) area[i] = 0.0;
    for (int f = 0; f < nf; f++) area[tri2bin[f]] += far_[f];
    #pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < ns; i++) {
        int f = sel[i];
        const double *a = V + 3 * F[3 * f], *b = V + 3 * F[3 * f + 1], *c = V + 3 * F[3 * f + 2];
        double ab[3], ac[3], N[3];
        for (int k = 0; k < 3; k++) { ab[k] = b[k] - a[k]; ac[k] = c[k] - a[k]; }
        N[0] = ab[1] * ac[2] - ab[2] * ac[1];
        N[1] = ab[2] * ac[0] - ab[0] * ac[2];
        N[2] = ab[0] * ac[1] - ab[1] * ac[0];
        double l = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        double n[3];
        for (int k = 0; k < 3; k++) { n[k] = l > 0.0 ? N[k] / l : 0.0; pos[3 * i + k] = cen[3 * f + k]; }
        int want = orient;
        if (orient && orient_list) {
            want = 0;
            for (int k = 0; k < n_orient; k++) want |= orient_list[k] == i;
        }
        if (want && l > 0.0) {
            double delta = 0.25 * sqrt(far_[f]);
            double qi[3], qo[3];
            for (int k = 0; k < 3; k++) { qi[k] = cen[3 * f + k] - delta * n[k]; qo[k] = cen[3 * f + k] + delta * n[k]; }
            double gi = orc_gwn_skip(V, F, nf, qi, f), go = orc_gwn_skip(V, F, nf, qo, f);
            if (!(gi > go)) for (int k = 0; k < 3; k++) n[k] = -n[k];
        }
        for (int k = 0; k < 3; k++) nrm[3 * i + k] = n[k];
    }
    free(cen);
    free(cenf);
    free(mind);
    free(far_);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
