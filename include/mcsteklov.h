/*
 * mcsteklov.h -- C ABI of the B300 Monte Carlo DtN / Steklov library.
 *
 * The library estimates the discrete Dirichlet-to-Neumann (DtN) stiffness
 * matrix Lambda of a triangle mesh from walk-on-spheres walks, as in
 * "Monte Carlo Steklov Operators for Large-Scale Geometry Processing in the
 * Wild" (Sec. 4.2, Alg. 2 "Final Interior DtN Estimator"; Sec. 4.3 exterior
 * estimator), and computes its smallest Steklov eigenpairs (Eq.
 * steklov-eigenproblem in Galerkin form Lambda psi = lambda M psi).
 *
 * Conventions
 *  - All functions return an mcs_status; 0 is success, negative values are
 *    errors, positive values are warnings.  mcs_last_error() returns a
 *    thread-local message for the last failing call on this thread.
 *  - "device" pointers are CUDA global-memory pointers on the current device;
 *    "host" pointers are ordinary CPU memory.  Each argument says which.
 *  - Output buffers are allocated by the caller, in sizes stated here.  The
 *    library allocates only inside mcs_build_bvh and mcs_build_bvh_batched
 *    (the meshes it owns until mcs_mesh_destroy; the builds' temporaries come
 *    from a stream-ordered pool the library keeps per device, up to 1 GiB
 *    reserved between builds) and nothing in the other calls: their scratch
 *    is the caller's workspace buffer (mcs_estimate_workspace_size bytes).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue their kernels on it and return without waiting,
 *    except where a host-side result (mcs_stats, a mesh handle) is requested:
 *    then the call synchronises that stream before returning.
 *  - Arguments are validated before any launch: invalid sizes, NULL required
 *    pointers, odd walk counts etc. return MCS_ERR_ARG and launch nothing.
 *    Failures detected on the device (traversal stack overflow) are reported
 *    through a device status word, read when stats are requested.
 *  - Results are deterministic: the same inputs, parameters and seed give
 *    bit-identical hit histograms on every run and every launch shape.
 */
#ifndef MCSTEKLOV_H
#define MCSTEKLOV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcs_mesh_s *mcs_mesh;

typedef enum {
    MCS_OK = 0,
    MCS_WARN_CAPPED = 1,            /* some walks hit max_steps (still counted) */
    MCS_WARN_NOT_CONVERGED = 2,     /* eigensolve: residual tolerance not met  */
    MCS_WARN_LOST = 3,              /* some walks were retired without a hit (stats.lost) */
    MCS_ERR_ARG = -1,
    MCS_ERR_CUDA = -2,
    MCS_ERR_OOM = -3,
    MCS_ERR_DEVICE = -4,            /* device status word set (see message)   */
    MCS_ERR_DEGENERATE = -5,        /* zero-extent mesh, non-finite input      */
    MCS_ERR_NO_INTERIOR_POINT = -6  /* exterior: no interior tangent ball      */
} mcs_status;

enum { MCS_FP32 = 32, MCS_FP64 = 64 };
enum { MCS_INTERIOR = 0, MCS_EXTERIOR = 1 };

/* Estimator parameters.  mcs_default_params() fills the paper's / the
 * design's defaults: eps 1e-3, theta0 = 2.5 deg (Sec. 5: cap of ~2.5 deg
 * around s excluded and the ball jump kernel importance sampled), 10
 * bisection iterations (Sec. 5), slack kappa 0.05 (vertex rows; 1e-6 is
 * used for sample rows when kappa < 0), max_steps 1024, rows with an
 * empty-ball radius below rho_min_factor * eps discarded (App. A item 2),
 * FP32 walks, interior, killing off (Sec. 5 footnote), seed 0. */
typedef struct {
    double eps;             /* WoS termination shell (inverted units for the exterior) */
    double cap_deg;         /* excluded cap half-angle theta0, degrees          */
    int bisect_iters;       /* tangent-ball bisection iterations                */
    double kappa;           /* tangent-ball slack; < 0: 0.05 vertex rows, 1e-6 sample rows */
    int max_steps;          /* closest-point queries per walk, >= 2             */
    double rho_min_factor;  /* discard rows whose empty radius < factor * eps   */
    int prec;               /* MCS_FP32 (walks in float, FP64 eps-shell) or MCS_FP64 */
    int domain;             /* MCS_INTERIOR or MCS_EXTERIOR                     */
    int origin_auto;        /* exterior: 1 = centre of the largest interior tangent ball
                               among rows 0, s, 2s, ... with s = ceil(n_rows / 256) */
    double origin[3];       /* exterior inversion centre when origin_auto == 0  */
    long long killing_walks;/* exterior: walks from the inverted origin (0 = killing off) */
    uint64_t seed;          /* Philox key                                       */
    int walks_per_row;      /* W, even (antithetic pairs)                       */
    int blocks_per_sm;      /* walk-kernel residency; 0 = library default       */
    int threads_per_block;  /* walk-kernel block size; 0 = library default      */
    int timing;             /* 1: time the phases with CUDA events (stats.phase_ms) */
    int count_work;         /* 1: count BVH nodes and triangles visited (slower; stats) */
    int queue_order;        /* walk queue schedule, bit 0: rows in the caller's order instead of
                               Z-order; bit 1 (batches): meshes by descending walk count.
                               Results do not depend on it (counter-based walks). */
    int bvh_layout;         /* BVH node layout of the walks' closest-point queries: 0 =
                               default (2), 2 = binary nodes (64 B), 4 = 4-wide nodes (the
                               binary tree collapsed two levels at a time, 128 B; needs
                               mcs_mesh_build_wide).  Same results either way. */
    int lanes_per_query;    /* with bvh_layout 4: 4 = a group of four lanes runs each walk,
                               lane r testing child r of each node; 0/1 = one lane per walk */
    int start_mode;         /* start points of the walks (interior estimates without the
                               nodal Lambda; for the variance comparison of Sec. 5):
                               0 = importance-sampled tangent ball (the estimator),
                               1 = cos(theta) uniform on the tangent ball outside the cap,
                               each walk weighted by q = |dB outside the cap| J^B / M
                               (outputs walk_w), 2 = the naive estimator (Alg. 1): one
                               uniform walk-on-spheres step from s - inset n, no cap,
                               row weight A_v / inset */
    double inset;           /* start_mode 2: the inset distance h (> 0)             */
} mcs_params;

/* Rows of the estimate.  Vertex rows: n_rows = nv, tri2bin = NULL, a walk's
 * exit column is the vertex of its exit triangle with the largest
 * barycentric weight.  Sample rows: tri2bin maps every triangle to its row. */
typedef struct {
    int n_rows;
    const double *pos;      /* device, n_rows x 3 row points s_v                */
    const double *nrm;      /* device, n_rows x 3 unit outward normals          */
    const double *area;     /* device, n_rows quadrature areas A_v              */
    const int32_t *tri2bin; /* device, nf, or NULL for vertex rows              */
} mcs_rows;

/* Outputs of mcs_estimate_dtn (device, caller-owned).  cap = min(W, n_rows).
 * The hit histogram is a padded CSR: row v holds hist_nnz[v] (bin, count)
 * pairs at offset v*cap, bins ascending, counts summing to W (0 for a
 * discarded row).  Lambda (n_rows x n_rows row-major FP64, optional) is the
 * assembled stiffness (Lambda32 its FP32 copy, rounded to nearest, for
 * consumers that work in FP32); omega (optional) the FP64 row weights; H0
 * (optional, exterior with killing walks) the killing-walk hit counts per
 * column. */
typedef struct {
    int32_t *hist_bin;      /* n_rows * cap                                     */
    int32_t *hist_cnt;      /* n_rows * cap                                     */
    int32_t *hist_nnz;      /* n_rows                                           */
    double *Lambda;         /* n_rows * n_rows, or NULL                         */
    double *omega;          /* n_rows, or NULL                                  */
    int32_t *H0;            /* n_rows, or NULL                                  */
    int32_t *exit_tri;      /* optional debug: n_rows * W exit triangle per walk (-1 discarded) */
    float *Lambda32;        /* optional: n_rows * n_rows FP32 copy of Lambda (needs Lambda) */
    double *exit_bary;      /* optional: n_rows * W * 3 barycentrics of each walk's exit point
                               on its exit triangle (F order of the vertices; 0 for a discarded
                               row or a walk without a hit); the input of the Galerkin estimator */
    double *walk_w;         /* optional: n_rows * W per-walk weights q (start_mode 1; 1 otherwise,
                               0 for a discarded row) */
} mcs_outputs;

typedef struct {
    long long walks, steps, capped;
    long long lost;         /* walks retired without a hit: exterior walks found at
                               |x~| > 2 / dist(o), i.e. in the inversion centre's own
                               component of a self-overlapping surface (they cannot
                               reach the exterior's boundary); interior walks farther
                               from the bounding-box centre than the box diagonal, i.e.
                               in the unbounded component (a row whose inward normal
                               points out); killing walks capped at x~ = 0.  Row sums
                               of H are W minus these */
    long long discarded_rows;
    long long killing_steps, killing_capped;
    double origin[3];       /* exterior inversion centre actually used          */
    double rmax;            /* tangent-ball radius clamp actually used          */
    int device_error;       /* 0 = none                                         */
    float phase_ms[4];      /* timing: row setup + tangent balls, walks, histogram, assembly */
    long long nodes_visited;/* count_work: BVH nodes whose child boxes were tested */
    long long tris_tested;  /* count_work: point-triangle tests                 */
} mcs_stats;

const char *mcs_last_error(void);
const char *mcs_version(void);
/* Instrumentation: kernels of this library enqueued on any stream since it
 * was loaded (a graph replay counts its captured library kernels; kernels
 * of the CUB sorts the library calls are not counted). */
unsigned long long mcs_launch_count(void);
void mcs_default_params(mcs_params *p);

/* Build the mesh: copies V (nv x 3 FP64) and F (nf x 3 int32, 0-based), in
 * host or device memory (detected), to the device; builds per-triangle
 * records in FP64 and FP32 and a linear BVH (Morton codes of triangle
 * centroids, radix sort, hierarchy of Karras 2012, bottom-up refit with
 * bounds rounded outward to float).  The paper uses the cuBQL BVH for WoS
 * closest-point queries (Sec. 5); this is the library's own.  Errors: ARG
 * (nv < 3, nf < 1, NULL), DEGENERATE (non-finite vertex, index out of range,
 * zero-extent bounding box), CUDA, OOM.  Synchronises `stream`. */
mcs_status mcs_build_bvh(const double *V, int nv, const int32_t *F, int nf, void *stream, mcs_mesh *out);
/* Build `count` meshes as mcs_build_bvh does (same records and hierarchy),
 * all enqueued on `stream` before one synchronisation: V[i], nv[i], F[i],
 * nf[i] describe mesh i; out[i] receives it.  On an error no mesh is
 * returned (all out[i] NULL), the status is that of the first failing mesh
 * and mcs_last_error names its index. */
mcs_status mcs_build_bvh_batched(int count, const double *const *V, const int *nv, const int32_t *const *F,
                                 const int *nf, void *stream, mcs_mesh *out);
void mcs_mesh_destroy(mcs_mesh m);
/* The mesh's 4-wide BVH (mcs_params.bvh_layout = 4): the binary tree
 * collapsed two levels at a time, built on request (allocates mesh-owned
 * device memory; synchronises `stream`).  mcs_mesh_has_wide tells whether it
 * exists (always true for one-triangle meshes). */
mcs_status mcs_mesh_build_wide(mcs_mesh m, void *stream);
int mcs_mesh_has_wide(mcs_mesh m);
int mcs_mesh_nv(mcs_mesh m);
int mcs_mesh_nf(mcs_mesh m);

/* Vertex rows (Alg. 2 rows on the lumped P1 basis): pos = V, nrm = unit sum
 * of incident face normals (b-a)x(c-a) in ascending face order (0 when the
 * sum vanishes: such a row is discarded), area = (incident face areas)/3.
 * Device outputs nv x 3, nv x 3, nv. */
mcs_status mcs_vertex_rows(mcs_mesh m, double *pos, double *nrm, double *area, void *stream);

/* Sample rows (point basis of Sec. 4.4; farthest-point sampling stands in
 * for blue noise): n samples over face centroids by greedy farthest-point
 * sampling from face 0; each face is owned by
 * its nearest sample (first selected on ties): tri2bin; a sample's area is
 * the total area of the faces it owns; its normal is the unit normal of the
 * sampled face, oriented (orient != 0) by the generalized winding number of
 * the other faces at x -/+ delta n, delta = sqrt(face area)/4 (App. A item 1):
 * the normal is kept when GWN(x - delta n) > GWN(x + delta n).  orient 3
 * sums the solid angles over the BVH, far nodes by their dipole term with a
 * certified bound on the remainder and on the float rounding; a row whose
 * gap does not exceed its bound is summed by brute force, so the decision is
 * the sign of the exact sum over the float-rounded triangles either way.
 * orient 2 sums every row by brute force (FP32).  orient 1 takes orient 3
 * when faces x rows >= 2^28 and orient 2 below (where the extra launches of
 * the hierarchical pass cost more than the brute-force sums).
 * Device outputs: sel n, pos n x 3, nrm n x 3, area n, tri2bin nf,
 * orient_gap n (optional: GWN(x - delta n) - GWN(x + delta n), within the
 * row's bound for rows decided by the hierarchical sum).  The
 * sampling runs in single precision on the float-rounded centroids (ties ->
 * lowest face id); meshes up to 2^18 faces use one block, larger ones a
 * thread-block cluster (16 CTAs where the device allows, else 8) that
 * exchanges candidates through distributed shared memory, and meshes beyond
 * the cluster's shared memory (~16M faces) a cooperative grid.
 * Synchronises `stream`. */
size_t mcs_sample_rows_workspace_size(mcs_mesh m, int n);
mcs_status mcs_sample_rows(mcs_mesh m, int n, int orient, int32_t *sel, double *pos, double *nrm, double *area,
                           int32_t *tri2bin, float *orient_gap, void *workspace, size_t workspace_bytes,
                           void *stream);

/* Sample rows of many meshes at once: each mesh's farthest-point sampling
 * runs as one block of a single launch (meshes in parallel), the rest as in
 * mcs_sample_rows, except that the hierarchical orientation of all meshes
 * runs in two launches and orient 1 chooses it when the batch's faces x rows
 * (summed over the meshes) reach 2^28.  The normals are those of
 * mcs_sample_rows (both passes decide only certified rows); orient_gap of a
 * row may come from the other pass.  Outputs per item as for mcs_sample_rows
 * (orient_gap optional).  workspace: device, 256-byte aligned, >=
 * mcs_sample_rows_batched_workspace_size.  Synchronises `stream`. */
typedef struct {
    mcs_mesh mesh;
    int n;
    int32_t *sel;
    double *pos, *nrm, *area;
    int32_t *tri2bin;
    float *orient_gap;
} mcs_sample_item;
size_t mcs_sample_rows_batched_workspace_size(const mcs_sample_item *items, int count);
mcs_status mcs_sample_rows_batched(const mcs_sample_item *items, int count, int orient, void *workspace,
                                   size_t workspace_bytes, void *stream);

/* Closest point of n query points (device, n x 3 FP64) by BVH traversal in
 * FP64 (prec 64) or FP32 (prec 32, points rounded to float), on the binary
 * (layout 2) or 4-wide (layout 4) nodes: squared distance, triangle id
 * (argmin of (d^2, id)), barycentrics.  Device outputs. */
mcs_status mcs_closest_points(mcs_mesh m, const double *P, int n, int prec, int layout, double *d2, int32_t *tri,
                              double *bary, void *stream);

/* Workspace bytes needed by mcs_estimate_dtn for these sizes. */
size_t mcs_estimate_workspace_size(mcs_mesh m, int n_rows, int walks_per_row, long long killing_walks);

/* The DtN estimator (Alg. 2; boxed interior estimator of Sec. 4.2; boxed
 * exterior estimator of Sec. 4.3 with the killing term):
 *   row setup   -- Morton (Z-order) row schedule (Sec. 5), tangent balls by
 *                  bisection (Sec. 5), discard rule (App. A item 2);
 *   walks       -- W per row from the empty tangent ball, start points
 *                  importance-sampled by J^B outside the cap, antithetic
 *                  pairs, Philox-4x32-10 counters (seed, row*W + walk, step);
 *                  WoS with BVH closest-point queries to the eps-shell;
 *                  exterior walks in the Kelvin-inverted domain;
 *   histogram   -- exit bins per row, warp-aggregated shared-memory counts
 *                  (up to 51200 rows), or the row's exits radix-sorted in
 *                  the block and run-length counted (more rows; then
 *                  walks_per_row <= 8192), into the padded CSR;
 *   assembly    -- W_vu = omega_v cf_u H_vu / W, Lambda = diag(Wsym 1) - Wsym
 *                  with Wsym = (W + W^T)/2 (+ diag of the killing measure).
 * workspace: device, >= mcs_estimate_workspace_size bytes, 256-byte aligned.
 * stats: host, optional; when given the call synchronises `stream`.
 * With stats requested, returns MCS_WARN_CAPPED when some walk was capped,
 * else MCS_WARN_LOST when some walk was retired without a hit (stats.lost). */
mcs_status mcs_estimate_dtn(mcs_mesh m, const mcs_rows *rows, const mcs_params *p, const mcs_outputs *out,
                            void *workspace, size_t workspace_bytes, mcs_stats *stats, void *stream);

/* ------------------------------------------------------------------ batches
 * Many meshes of uneven size and row count in one persistent walk launch
 * (the paper estimates one shape at a time; its large-scale preprocessing
 * runs shapes one after another, Sec. 6).  Each mesh gets its row setup and
 * tangent balls; then ONE walk launch serves all meshes' walks from one
 * global queue (meshes in table order, each mesh's row walks in its row
 * order, then its killing walks); then each mesh's histogram and assembly.
 * A mesh's results are bit-identical to mcs_estimate_dtn on that mesh with
 * the same parameters, domain and seed.  The shared parameters (eps, W,
 * precision, killing_walks, launch shape...) come from one mcs_params; its
 * domain, origin and seed fields are ignored in favour of the item's. */
typedef struct {
    mcs_mesh mesh;
    mcs_rows rows;
    int domain;             /* MCS_INTERIOR or MCS_EXTERIOR                     */
    int origin_auto;        /* exterior: 1 = automatic inversion centre         */
    double origin[3];       /* exterior centre when origin_auto == 0            */
    uint64_t seed;          /* Philox key of this mesh's walks                  */
    mcs_outputs out;        /* as for mcs_estimate_dtn (device, caller-owned)   */
} mcs_batch_item;

/* Workspace bytes of a batch (device, 256-byte aligned). */
size_t mcs_estimate_batched_workspace_size(const mcs_batch_item *items, int n, int walks_per_row);
/* Enqueues the batch on `stream`.  total (host, optional): the launch's
 * counters summed over meshes; per_item (host, optional, n entries): each
 * mesh's counters and status fields.  When either is given the call
 * synchronises `stream` and returns the worst status over the meshes
 * (errors before warnings); the error text names the first failing meshes. */
mcs_status mcs_estimate_batched(const mcs_batch_item *items, int n, const mcs_params *p, void *workspace,
                                size_t workspace_bytes, mcs_stats *total, mcs_stats *per_item, void *stream);

/* The batch captured once into a CUDA graph (on a private stream, thread-
 * local capture mode) and instantiated: mcs_graph_launch replays every
 * kernel of mcs_estimate_batched with one host call.  The graph holds the
 * device pointers of the items, outputs and workspace given here: they must
 * stay valid, and the inputs may change in place between launches (not the
 * sizes).  mcs_graph_stats synchronises `stream` and reads the counters of
 * the last finished launch.  With p->timing set, the graph records CUDA
 * events around its phases at every replay, and mcs_graph_stats also returns
 * the last replay's phase times (phase_ms: setup, walks, histogram and
 * assembly).  A graph may not be launched concurrently with itself or with
 * another call that uses the same workspace. */
typedef struct mcs_graph_s *mcs_graph;
mcs_status mcs_graph_create(const mcs_batch_item *items, int n, const mcs_params *p, void *workspace,
                            size_t workspace_bytes, mcs_graph *out);
mcs_status mcs_graph_launch(mcs_graph g, void *stream);
mcs_status mcs_graph_stats(mcs_graph g, mcs_stats *total, mcs_stats *per_item, void *stream);
size_t mcs_graph_nodes(mcs_graph g);
void mcs_graph_destroy(mcs_graph g);

/* Autotuner of the walk launch.  Runs the batch's row setup, then times the
 * walk kernel on a sample (every s-th row of every mesh's row schedule,
 * s = floor(1 / sample_fraction), lowered so that the sample holds at least
 * 32 walks per resident lane of the default launch, or the whole batch when
 * it has fewer: a shorter sample is dominated by the launch's tail and
 * misranks the layouts; no killing walks) for the row order of
 * the queue (a batch of several meshes always dispenses them longest first,
 * queue_order bit 1: its benefit, a shorter tail, grows with the walks per
 * mesh and does not show in the sample), the BVH node layouts (when p->bvh_layout is 0),
 * candidate block sizes (64, 128 threads), each at the largest residency the
 * kernel allows (a smaller one looks better in the sample's tail, with few
 * walks per SM, than in the full launch), by coordinate search in that
 * order; each trial takes the best of three runs, and a candidate replaces
 * the incumbent only when it is more than 5% faster (smaller differences are
 * within the sample's run-to-run noise).  tuned (host) = p with bvh_layout, lanes_per_query,
 * threads_per_block, blocks_per_sm and queue_order set.  trials (host, optional) receives up to
 * max_trials entries, n_trials their count.  Synchronises `stream`.  The
 * workspace and outputs are those of the batch; their contents are left
 * undefined (the estimate rewrites them). */
typedef struct {
    int threads_per_block, blocks_per_sm, queue_order, bvh_layout, lanes_per_query;
    float ms;               /* walk-kernel time of the sample (best of 3)       */
} mcs_tune_trial;
mcs_status mcs_autotune_walks(const mcs_batch_item *items, int n, const mcs_params *p, void *workspace,
                              size_t workspace_bytes, double sample_fraction, mcs_params *tuned,
                              mcs_tune_trial *trials, int max_trials, int *n_trials, void *stream);

/* Allocation-free estimate.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need an
 * estimate -- code running inside a memory pool or arena it does not own, a
 * custom allocator that forbids cudaMalloc in a critical section, or a
 * process that must not change its allocator state while the device is full.
 * It runs mcs_estimate_dtn with its scratch taken from a fixed 32 MiB array
 * that the library reserves on every GPU where it is loaded (held until the
 * process exits); it calls no cudaMalloc, cudaFree or allocating library
 * routine, and creates no events (phase timing is off).  The caller still
 * passes rows, parameters and outputs as for mcs_estimate_dtn.
 *  - Estimates whose scratch (mcs_estimate_workspace_size) exceeds
 *    mcs_estimate_dtn_noalloc_capacity() bytes are rejected with MCS_ERR_ARG.
 *  - CUDA loads a library's code and device arrays lazily, at first use, and
 *    loading reserves device memory.  mcs_build_bvh (which allocates the
 *    mesh anyway) therefore loads this array and every kernel the estimate
 *    launches on the current device, so that a call on a mesh built earlier
 *    in the same CUDA context allocates nothing.  Each call looks up the
 *    array's device address (cudaGetSymbolAddress) with the mesh's device
 *    current; make the first call before capturing a stream.
 *  - The walks run in the caller's row order (queue_order bit 0 is set): the
 *    Z-order schedule would need a library sort.  The results are those of
 *    mcs_estimate_dtn, which do not depend on the schedule.
 *  - All calls share the one array, which keeps the last call's contents;
 *    every part the estimate reads is rewritten or cleared by the call itself.
 *    Calls that overlap on the GPU (other streams, other threads) race on it:
 *    serialise them. */
size_t mcs_estimate_dtn_noalloc_capacity(void);
mcs_status mcs_estimate_dtn_noalloc(mcs_mesh m, const mcs_rows *rows, const mcs_params *p, const mcs_outputs *out,
                                    mcs_stats *stats, void *stream);

/* Steklov eigensolve (Eq. steklov-eigenproblem, Galerkin form Lambda psi =
 * lambda M psi with M = diag(mass); smallest k pairs, Sec. 4.4 / Sec. 5).
 * Chebyshev-filtered subspace iteration on a block of m = k + 32 vectors
 * (rounded up to 16, at most 160): filter products A*Y on the tensor cores
 * (tcgen05 kind::tf32, operands split into tf32 high/low parts), or, for a
 * sparse A (histogram rows of a large surface reach few bins), on A in CSR
 * with FP32 values, one fused SIMT kernel per filter term; FP64
 * CholeskyQR2 orthonormalisation (a shifted CholeskyQR first on the start block, and after a filter
 * whose block has lost numerical rank), Rayleigh-Ritz with a
 * parallel Jacobi on the block, Ritz values as FP64 Rayleigh quotients. */
typedef struct {
    int degree;             /* Chebyshev filter degree per iteration (<= 256; 0, the default:
                               48 with the dense product, 96 with the sparse one); halved
                               (down to 8) after two iterations that add no converged pair */
    int max_iters;          /* outer iterations (60)                             */
    double tol;             /* residual |A x - theta x| <= tol * upper bound (1e-5) */
    int product;            /* operator of the filter products: 0 chooses (the sparse one when
                               at most one entry of A in 32 is nonzero), 1 dense tf32-split
                               tensor-core product, 2 sparse (CSR, FP32 values and sums) */
} mcs_eig_params;
typedef struct {
    int iterations, converged, block, tc_products;  /* tc_products: filter and Rayleigh-Ritz
                                                       products of either kind */
    double upper_bound, max_residual;
    int device_error;
    int product;            /* the operator used: 1 dense, 2 sparse                          */
    long long nnz;          /* nonzeros of A (entries that round to a nonzero float)         */
    int jacobi_sweeps;      /* Jacobi sweeps of the Rayleigh-Ritz steps, summed              */
} mcs_eig_stats;
void mcs_default_eig_params(mcs_eig_params *p);
size_t mcs_steklov_workspace_size(int n, int k);
/* Lambda: device n x n FP64 symmetric (row-major); mass: device n (> 0);
 * evals: k FP64, host or device (ascending); evecs: device n x k FP64
 * row-major psi (M-orthonormal), or NULL; workspace: device, 256-byte
 * aligned, >= mcs_steklov_workspace_size(n, k).  Requires 16 <= n and
 * 1 <= k <= min(128, n/2 - 1).  Synchronises `stream` (the convergence test
 * reads the residuals on the host each iteration).  Returns
 * MCS_WARN_NOT_CONVERGED when max_iters was reached first. */
mcs_status mcs_steklov_modes(const double *Lambda, const double *mass, int n, int k, double *evals, double *evecs,
                             void *workspace, size_t workspace_bytes, const mcs_eig_params *params,
                             mcs_eig_stats *stats, void *stream);
/* Galerkin estimator (Sec. 4.4, mesh-based Galerkin basis; boxed
 * estimators Eq. main-estimator and Eq. main-exterior-estimator with
 * d(s,t) = b(s) - b(t), b evaluated by barycentric interpolation).
 *
 * mcs_cotan_laplacian: the dense cotangent Laplacian of the mesh, L[a][b] =
 * -(cot alpha + cot beta)/2 over the faces sharing edge (a, b), L[a][a] = -sum
 * of the row; device nv x nv FP64 row-major (overwritten).  Its smallest
 * generalized eigenpairs with the lumped vertex areas (mcs_steklov_modes with
 * mass = the vertex-row areas) are the paper's default basis Phi.
 *
 * mcs_galerkin_dtn: S = Phi^T Lambda_bary Phi (device K x K FP64), where
 * Lambda_bary = sum over recorded walks of w (e_s - beta_t)(e_s - beta_t)^T:
 * e_s the row point's nodal coefficients (vertex rows: its vertex; sample
 * rows: row_face[v]'s vertices, 1/3 each), beta_t the exit barycentrics on the
 * exit triangle, w = omega_v / (2 W) (the boxed estimators' factor 1/2)
 * times |t - o| at the hit point t for an
 * exterior estimate (o = origin, host 3 doubles).  Inputs from an estimate
 * with exit_tri and exit_bary recorded (mcs_outputs): omega n_rows, exit_tri
 * and exit_bary n_rows x W (x 3).  Killing walks (exterior, H0 with
 * killing_walks > 0, optional) enter lumped at their bin: 4 pi |p - o| H0 /
 * N0.  walk_w (optional, n_rows x W): per-walk weights multiplying w
 * (start_mode 1).  form 0: the jump form above; form 1 (interior; start_mode
 * 2): the naive estimator's (Alg. 1) symmetrised
 * w [e_s (e_s - beta_t)^T + (e_s - beta_t) e_s^T] / 2 with w = omega_v / W.
 * Phi: device nv x K FP64 row-major, M-orthonormal; K a multiple of 16
 * in [16, 160]; nv >= 16.  Lambda_bary: optional device nv x nv output, else
 * held in the workspace (own_lambda = 1 in the size query).  Lambda_bary is
 * assembled with FP64 atomics (reproducible to rounding); Lambda_bary Phi
 * runs on the tensor cores (split tf32, FP32-level accuracy).  Synchronises
 * `stream`.
 *
 * mcs_galerkin_modes: eigenpairs of the symmetric K x K matrix S (with Phi
 * M-orthonormal, the Galerkin Steklov problem S c = lambda c), cyclic Jacobi
 * in FP64: evals device K (ascending), coeffs device K x K (eigenvectors in
 * columns), psi optional device n x k = Phi coeffs[:, :k] (the Steklov modes
 * on the vertices).  2 <= K <= 160.  Asynchronous on `stream`. */
mcs_status mcs_cotan_laplacian(mcs_mesh m, double *L, void *stream);
size_t mcs_galerkin_workspace_size(mcs_mesh m, int K, int own_lambda);
mcs_status mcs_galerkin_dtn(mcs_mesh m, const mcs_rows *rows, const int32_t *row_face, const double *omega,
                            const int32_t *exit_tri, const double *exit_bary, const double *walk_w, int form,
                            int walks_per_row, int exterior,
                            const double *origin, const int32_t *H0, long long killing_walks, const double *Phi,
                            int K, double *S, double *Lambda_bary, void *workspace, size_t workspace_bytes,
                            void *stream);
mcs_status mcs_galerkin_modes(const double *S, int K, int k, const double *Phi, int n, double *evals, double *coeffs,
                              double *psi, void *stream);

/* mcs_galerkin_project: S = Phi^T Lambda Phi (device K x K FP64) for any
 * symmetric device n x n FP64 Lambda (e.g. the point-basis matrix of
 * mcs_point_galerkin_lambda) and device n x K FP64 Phi; K a multiple of 16 in
 * [16, 160], n >= 16.  Lambda Phi runs on the tensor cores (split tf32,
 * FP32-level accuracy).  workspace: device, 256-byte aligned,
 * >= mcs_galerkin_project_workspace_size(n, K) (0 for invalid sizes).
 * Synchronises `stream`. */
size_t mcs_galerkin_project_workspace_size(int n, int K);
mcs_status mcs_galerkin_project(const double *Lambda, const double *Phi, int n, int K, double *S, void *workspace,
                                size_t workspace_bytes, void *stream);

/* Point-based Galerkin basis (Sec. 4.4 "Point-based Galerkin basis";
 * appendix "Point-based k-NN Interpolator").  P: device n_points x 3 FP64
 * surface points (e.g. farthest-point sample rows), NP: their unit normals
 * (device n_points x 3).  Each call builds a uniform grid over P in its
 * workspace (device, 256-byte aligned, >= mcs_points_workspace_size(n_points))
 * and synchronises `stream` once (to read the grid's size); the rest is
 * asynchronous on `stream`.  All FP64.
 *
 * mcs_point_knn: the k (1..32) nearest points of each query Q (device
 * n_queries x 3): squared distances ((dx dx + dy dy) + dz dz), d = q - p,
 * ascending, equal distances by the smaller index (exact and reproducible).
 * exclude_self = 1 (queries = the points) skips each query's own point.
 * Outputs (each optional, at least one): idx device n_queries x k int32, d2
 * device n_queries x k, w device n_queries x k bilateral weights
 * (needs NP, NQ = the query normals, sigma, tau_n > 0):
 * w_i proportional to exp(-|q - x_i|^2 / (2 sigma^2)) exp(-(1 - <n_q, n_i>) / tau_n),
 * normalised to sum 1 (the paper's values: sigma 0.025, tau_n 0.8, k 8).
 *
 * mcs_point_laplacian: the point-cloud Laplacian.  Each point's k_nbr
 * (3..32, < n_points) nearest other points are projected on its tangent plane
 * (frame e1 = n x a / |n x a|, a the axis of n's smallest |component|,
 * e2 = n x e1); the Voronoi cell of the point among them (a box of half-size
 * 2 max |u_j| cut by the bisector half-planes) gives the weight
 * w_ij = |cell edge on the (i, j) bisector| / |u_j|.  L (device n x n,
 * overwritten): L_ij = -(w_ij + w_ji) / 2, L_ii = -sum_{j != i} L_ij.
 * nbr / nbr_w (device n x k_nbr): the neighbours and their local weights;
 * cell_area (optional, device n): the local cell areas.
 *
 * mcs_point_galerkin_lambda: the Galerkin matrix over the points (device
 * n_points x n_points, overwritten) from an estimate whose rows were the
 * points themselves (row r starts at P[r]) with exit_tri / exit_bary
 * recorded: sum over walks of w (b_s - b_t)(b_s - b_t)^T, b_s the
 * interpolator at P[r] (normal NP[r]), b_t at the exit point (normal of the
 * exit face), w = omega_r / (2 W), times |t - o| for an exterior estimate
 * (origin host 3 doubles).  Killing walks (exterior, H0 with killing_walks >
 * 0, optional) add 4 pi |P[r] - o| H0[r] / N0 b_s b_s^T.  FP64 atomics
 * (reproducible to rounding).  Its smallest generalised eigenpairs with the
 * point areas give Phi for mcs_galerkin_project. */
size_t mcs_points_workspace_size(int n_points);
mcs_status mcs_point_knn(const double *P, const double *NP, int n_points, const double *Q, const double *NQ,
                         int n_queries, int k, double sigma, double tau_n, int exclude_self, int32_t *idx, double *w,
                         double *d2, void *workspace, size_t workspace_bytes, void *stream);
mcs_status mcs_point_laplacian(const double *P, const double *NP, int n_points, int k_nbr, double *L,
                               double *cell_area, int32_t *nbr, double *nbr_w, void *workspace,
                               size_t workspace_bytes, void *stream);
mcs_status mcs_point_galerkin_lambda(mcs_mesh m, const double *P, const double *NP, int n_points,
                                     const double *omega, const int32_t *exit_tri, const double *exit_bary,
                                     int walks_per_row, int exterior, const double *origin, const int32_t *H0,
                                     long long killing_walks, int k, double sigma, double tau_n, double *Lambda_P,
                                     void *workspace, size_t workspace_bytes, void *stream);

/* Steklov heat (Sec. 5, Eq. steklovHeat, solved in the eigenbasis by Eq.
 * spectralSteklovHeat): for each time t and each channel column of u0,
 *   u_t = sum_j exp(-lambda_j t) a_j psi_j,  a_j = psi_j^T M u_0,
 * with the interior or exterior eigenpairs of mcs_steklov_modes.
 * evals: device k FP64; evecs: device n x k FP64 row-major, M-orthonormal;
 * mass: device n; u0: device n x c row-major (c channels); times: device nt;
 * out: device nt x n x c row-major.  1 <= k <= 128.  workspace: device,
 * 256-byte aligned, >= mcs_steklov_heat_workspace_size(n, k, c).  FP64, sums
 * in a fixed order (bitwise reproducible).  Asynchronous on `stream`. */
size_t mcs_steklov_heat_workspace_size(int n, int k, int c);
mcs_status mcs_steklov_heat(const double *evals, const double *evecs, const double *mass, int n, int k,
                            const double *u0, int c, const double *times, int nt, double *out, void *workspace,
                            size_t workspace_bytes, void *stream);
/* Heat kernel signature of the Steklov eigenpairs (Sun et al. 2009; the
 * basis-invariant comparison of spectra in Sec. 5, Fig. hks_comparison):
 *   out[t][x] = sum_j exp(-lambda_j t) psi_j(x)^2.
 * evals: device k; evecs: device n x k row-major; times: device nt; out:
 * device nt x n.  1 <= k <= 128.  FP64, fixed summation order.  Needs no
 * workspace.  Asynchronous on `stream`. */
mcs_status mcs_hks(const double *evals, const double *evecs, int n, int k, const double *times, int nt, double *out,
                   void *stream);
/* Test hook: Zt = (A X)^T through the same tensor-core product, for a
 * symmetric A (device n x n FP64) and Xt (device m x n FP64, m a multiple
 * of 16 in [16, 160]); Zt device m x n FP64. */
size_t mcs_tc_symm_product_workspace_size(int n, int m);
mcs_status mcs_tc_symm_product(const double *A, const double *Xt, int n, int m, double *Zt, void *workspace,
                               size_t workspace_bytes, void *stream);

/* Test hook: Philox-4x32-10 words for counters (i_lo, i_hi, c2, c3),
 * i = start .. start+n-1, key (k0, k1); device output n x 4. */
mcs_status mcs_philox_words(uint64_t start, uint64_t n, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                            uint32_t *out, void *stream);

/* Measurement probes (the paper has no counterpart): the hardware ceilings
 * the walk kernel's roofline is stated against, measured on the running GPU.
 * The caller times each call with CUDA events on `stream`.
 *  - mcs_probe_l2_read: every SM streams `reps` passes over the device
 *    buffer buf (bytes, a multiple of 16, 16-byte aligned) with loads that
 *    bypass L1 (ld.global.cg); a buffer below the L2 size measures L2 read
 *    bandwidth (bytes * reps / time).  sink: device 8 bytes (written only
 *    to keep the loads).
 *  - mcs_probe_fma32 / mcs_probe_fma64: 148-SM-filling grid, every thread
 *    runs 8 independent fused multiply-add chains of `iters` steps; the
 *    instruction rate is threads * 8 * iters / time (2 FLOP each).
 *    mcs_probe_threads() is the thread count of that grid.  out: device
 *    4 bytes (FP32) / 8 bytes (FP64), written only to keep the chains.
 * Invalid sizes give MCS_ERR_ARG; asynchronous on `stream`. */
mcs_status mcs_probe_l2_read(const void *buf, size_t bytes, int reps, unsigned long long *sink, void *stream);
mcs_status mcs_probe_fma32(int iters, float *out, void *stream);
mcs_status mcs_probe_fma64(int iters, double *out, void *stream);
long long mcs_probe_threads(void);

#ifdef __cplusplus
}
#endif
#endif
