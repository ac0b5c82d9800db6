/*
 * htlr.h -- C ABI of the GB300 (sm_103a) HTLR library.
 *
 * Hierarchical Tucker low-rank (HTLR) matrices, after Li & Liu, "Hierarchical Tucker
 * Low-Rank Matrices: Construction and Matrix-Vector Multiplication" (arXiv 2508.05958).
 * The library builds the HTLR representation of the Nystrom operator
 *
 *     f_i = a(x_i) u_i + sum_j K_ij w_j u_j,                      (eq. (1.3), §3.3)
 *     K_ij = k(x_i, x_j) (j != i),  K_ii w_i = int_{Omega_i} k(x_i, y) dy   (eq. (1.4))
 *
 * on a tensor grid of [0,1]^d (d = 2 or 3, N = n^d points, w_j = |Omega_j| = h^d on the
 * uniform grid of Example 2.1) and applies it to vectors (HMultVec, Algorithm 2).
 *
 * Conventions shared by every call:
 *   - Points are numbered in natural order i_1 + n i_2 + n^2 i_3 (first index fastest, §2.1).
 *   - Vectors are N x nrhs, column-major, leading dimension N, FP64.
 *   - All calls return HTLR_OK (0) or a negative htlr_status; no C++ exception crosses the
 *     ABI.  On failure htlr_last_error() returns a message for the calling thread.
 *   - Device work is enqueued on the handle's CUDA stream; calls that take device
 *     pointers return before the work finishes.
 *   - Every call is made on the CUDA device that was current at construction.
 */
#ifndef HTLR_H
#define HTLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
    HTLR_OK = 0,
    HTLR_EINVAL = -1,        /* invalid argument (the message names it) */
    HTLR_ENOMEM = -2,        /* footprint above the HBM limit, checked before allocating */
    HTLR_ECUDA = -3,         /* a CUDA runtime call failed (message has the CUDA error) */
    HTLR_EUNSUPPORTED = -4,  /* valid, but not supported by this library (e.g. SHARED storage
                                on a non translation-invariant setting) */
    HTLR_ETIMEOUT = -5,      /* a bounded device wait ran out */
    HTLR_EDEVICE = -6        /* a kernel reported an internal check failure */
} htlr_status;

/* Kernel functions k(x, y), r = |x - y|.  The paper's experiments use the Gaussian and the
 * single-layer potential (§5): SLP is LOG with scale -1/(2 pi) in 2D and INV_R with scale
 * 1/(4 pi) in 3D. */
typedef enum {
    HTLR_K_LOG = 0,    /* scale * log r */
    HTLR_K_INV_R = 1,  /* scale / r */
    HTLR_K_EXP_R = 2,  /* scale * exp(-r) */
    HTLR_K_GAUSS = 3,  /* scale * exp(-r^2 / (2 param^2)), param = sigma */
    HTLR_K_POLY = 4,   /* scale * prod_l (x_l - y_l + 2 + l/2)^param, l = 0..d-1: a test
                          kernel of per-dimension degree param (integer 0..16) */
    HTLR_K_CONST = 5   /* scale */
} htlr_kernel_type;

typedef struct {
    int type;        /* htlr_kernel_type */
    double scale;
    double param;
} htlr_kernel;

typedef enum {
    HTLR_GRID_UNIFORM = 0,  /* x_i = (i + 1/2)/n, cells [i/n, (i+1)/n] (Example 2.1) */
    HTLR_GRID_TENSOR = 1    /* per-dimension coordinates and cell edges given (§3.3) */
} htlr_grid_type;

typedef struct {
    int type;              /* htlr_grid_type */
    const double *coords;  /* TENSOR: d*n host doubles, coords[l*n + i], increasing in (0,1) */
    const double *edges;   /* TENSOR: d*(n+1) host doubles, cell of line i in dimension l is
                              [edges[l*(n+1)+i], edges[l*(n+1)+i+1]], edges 0 and 1 at the ends */
    const double *a;       /* host array of N values a(x_i) in natural order, or NULL: a = 0 */
} htlr_grid;

/* How admissible-block cores and inadmissible blocks are held in HBM. */
typedef enum {
    HTLR_STORE_AUTO = 0,    /* STORED if it fits the limit, else SHARED when allowed */
    HTLR_STORE_STORED = 1,  /* one core per admissible block and one dense matrix per
                               inadmissible block, as Algorithm 1 builds them */
    HTLR_STORE_SHARED = 2,  /* uniform grid + translation-invariant kernel: blocks with the
                               same level and box offset are equal, so one core (and one
                               dense block) per (level, offset) is kept */
    HTLR_STORE_GENERATED = 3 /* cores per (level, offset) as SHARED; the inadmissible blocks
                               are not stored but recomputed from the kernel function in
                               every matvec.  Always used on tensor grids, whose dense
                               blocks differ from pair to pair */
} htlr_storage;

/* Arithmetic of the far-field (core) and near-field (dense block) products. */
typedef enum {
    HTLR_PREC_FP64 = 0,  /* FP64 blocks and FP64 fused multiply-adds */
    HTLR_PREC_DF64 = 1,  /* FP64 blocks held as float pairs (hi + lo, 48-bit significand) and
                            products formed with error-free FP32 transformations; results
                            within ~1e-14 of FP64.  Entries must lie within FP32 range,
                            |x| in [1e-30, 1e30], for that accuracy */
    HTLR_PREC_FP32 = 2,  /* FP32 blocks, products and accumulation.  Unit roundoff 6e-8;
                            measured 7e-9 to 1.5e-6 relative on the full-size operators,
                            more where the result cancels (random u against a smooth
                            kernel).  A generated near field sums each source leaf apart
                            and then adds the leaf sums */
    HTLR_PREC_BF16X6 = 3, /* tensor cores (tcgen05): operands split into three BF16 terms,
                            the six products a_i b_j with i + j <= 4 (1-based) accumulated
                            in FP32 tensor memory; the many-right-hand-side path, 64 RHS at
                            a time.  The tensor cores' FP32 accumulation truncates each
                            addition, so with SHARED blocks the accumulation runs in short
                            segments (tc_segment) that start fresh with the small cross
                            products, whose sums are added in FP32 registers and flushed to
                            FP64 every tc_flush segments.  STORED blocks are refused
                            (HTLR_EUNSUPPORTED); AUTO storage resolves to SHARED.  A BF16X6
                            far field goes with a BF16X6, generated (FP64, FP32 or TF32X3),
                            or held FP64/df64/FP32 near field; a BF16X6 near field needs a
                            BF16X6 far field */
    HTLR_PREC_TF32X3 = 4 /* near field only, generated (tensor grids, HTLR_STORE_GENERATED,
                            or AUTO storage, which then generates it): kernel values
                            computed per point pair in FP32 and written into tensor memory
                            as two TF32 terms (nearest, then the exact rest), w_j u_j as two
                            TF32 terms, the three products a2 b1, a1 b2, a1 b1 (tcgen05
                            kind::tf32), 16 right-hand sides per pass; FP32 accumulation in
                            segments of two 16-source stages that start fresh with the cross
                            products, summed in FP32 and flushed to FP64 every 16 segments.
                            Measured within 1e-6 of the FP64 oracle on every kernel type */
} htlr_precision;

typedef struct {
    int storage;       /* htlr_storage (default AUTO) */
    int orth;          /* 1: QR-orthonormalise the factors (Algorithm 1), 0: keep the
                          interpolation factors; -1: default (1 on the uniform grid, 0 on
                          tensor grids, which support only 0) */
    int quad_order;    /* Gauss-Legendre points per dimension and sub-box for the diagonal
                          integral (default 16, range 1..64) */
    void *stream;      /* cudaStream_t for construction and matvecs (NULL: default stream) */
    size_t hbm_limit;  /* maximum bytes the handle may allocate (0: 90% of free memory) */
    int far_precision;   /* htlr_precision of the admissible blocks (default FP64) */
    int near_precision;  /* htlr_precision of the inadmissible blocks (default FP64) */
    int tc_segment;      /* BF16X6 with SHARED blocks: K steps of 16 columns per tensor-memory
                            segment (0: default 4).  A
                            segment starts from a fresh accumulator; its cross products
                            (a3b1, a2b2, a1b3, a2b1, a1b2) are accumulated first, while the
                            sum is small, and the leading products a1b1 last, because the
                            tensor cores' FP32 accumulation truncates every addition (about
                            2^-24 of the running sum, biased toward zero) */
    int tc_flush;        /* BF16X6 with SHARED blocks: segments summed in FP32 registers before
                            they are added to the FP64 result (0: default 32) */
    long long tc_wait_cycles; /* limit, in SM clock cycles, of every bounded wait inside the
                            tensor-core kernels (a copy, an MMA or a drain that does not
                            complete): 0 selects the default 4e9 (about 2 s at 2 GHz).  When
                            a wait runs out the kernel stops its work, lets what it already
                            issued complete, releases its tensor memory and returns; the
                            matvec's result is then invalid and htlr_sync (or the next
                            synchronous call) returns HTLR_ETIMEOUT */
} htlr_options;

/* Statistics of a constructed operator (htlr_info). */
#define HTLR_MAX_LEVELS 16
typedef struct {
    int d, n, levels;                 /* levels L: the leaves are at level L */
    int p, p_eff_leaf;                /* Tucker rank p and its value after QR at the leaves */
    int storage;                      /* the htlr_storage actually used */
    int64_t far_per_level[HTLR_MAX_LEVELS];  /* admissible leaves (TLR blocks) per level */
    int64_t near_blocks;              /* inadmissible leaves (dense blocks) */
    int64_t unique_cores;             /* cores held (== far blocks for STORED) */
    int64_t unique_near;              /* dense blocks held */
    double paper_storage_doubles;     /* storage of the paper's layout: per far block p_eff^{2d}
                                         core + factors sum_l (|tau_l| + |sigma_l|) p_eff, per
                                         near block |tau| |sigma| (Prop. 3.4/3.5, §5) */
    size_t bytes_cores, bytes_near, bytes_factors, bytes_work, bytes_total;
    double diag_value;                /* K_ii w_i on the uniform grid (eq. (1.4)) */
    int far_precision, near_precision;  /* htlr_precision in use */
    int tc_grouped;                   /* BF16X6 block lists on the target-grouped tensor-core
                                         kernel (SHARED): bit l for far level l, bit 31 for
                                         the inadmissible leaves */
    int64_t near_point_pairs;         /* sum over inadmissible leaves of |tau| |sigma| */
} htlr_stats;

typedef struct htlr_handle htlr_handle;

/*
 * htlr_construct -- Construct (Algorithm 1) on the current device.
 *   H      out: new handle; owns every device allocation it makes.
 *   k      kernel function (copied).
 *   d      2 or 3.
 *   n      points per dimension; n = leaf * 2^L with L >= 1 and L < HTLR_MAX_LEVELS.
 *   grid   grid description (copied); NULL means the uniform grid with a = 0.
 *   leaf   points per dimension in a leaf box (the leaf test |tau| <= N_0 of §2.2 with
 *          N_0 = leaf^d).
 *   r      Tucker rank p: Chebyshev points per dimension (1..16).
 *   eta    strong admissibility max(diam) <= eta * dist (Def. 2.3) on the geometric tree
 *          cells; eta <= 0 selects weak admissibility (Def. 2.2).
 * Errors: HTLR_EINVAL (bad argument), HTLR_ENOMEM (footprint over the limit, nothing
 * allocated), HTLR_EUNSUPPORTED, HTLR_ECUDA.  *H is NULL on failure.
 * Synchronous: returns after the construction kernels finished.
 */
int htlr_construct(htlr_handle **H, const htlr_kernel *k, int d, int n,
                   const htlr_grid *grid, int leaf, int r, double eta);

/* htlr_construct with options (o may be NULL for defaults). */
int htlr_construct_ex(htlr_handle **H, const htlr_kernel *k, int d, int n,
                      const htlr_grid *grid, int leaf, int r, double eta,
                      const htlr_options *o);

/*
 * htlr_matvec -- f = A u (HMultVec, Algorithm 2, started from the root with f = 0).
 *   u, f   device pointers, N x nrhs column-major FP64, caller-owned; must not overlap.
 *   nrhs   >= 1.
 * Asynchronous on the handle's stream.  f is overwritten.
 */
int htlr_matvec(const htlr_handle *H, const double *u, double *f, int nrhs);

/*
 * htlr_matvec_host -- f = A u with HOST arrays: copies u to the device, applies, copies f
 * back, all on the handle's stream, and returns after f is in host memory.  Uses device
 * staging buffers owned by the handle (grown on demand).
 */
int htlr_matvec_host(htlr_handle *H, const double *u_host, double *f_host, int nrhs);

/*
 * htlr_matvec_timed -- htlr_matvec that also measures, with CUDA events recorded on the
 * handle's stream, the device time of each stage: stage_ms[0] upward contractions,
 * [1] block streaming (cores and held dense blocks, on CUDA or tensor cores, with the
 * packing of their operands), [2] the near field in its own launches: generated (on the
 * CUDA cores, or on the tensor cores for TF32X3, packing of w u included), or held beside
 * a tensor-core far field, [3] per-row reductions, [4] downward
 * expansion + output.  Times are summed over RHS chunks.  Synchronous
 * (waits for the stream).  stage_ms: host array of HTLR_NUM_STAGES floats.
 */
#define HTLR_NUM_STAGES 5
int htlr_matvec_timed(const htlr_handle *H, const double *u, double *f, int nrhs,
                      float *stage_ms);

/*
 * htlr_matvec_noalloc -- f = A u, like htlr_matvec, but without any device allocation:
 * its scratch (the per-level contracted tensors W and H, the partial sums of the block
 * stream and a small task table) is taken from one fixed array of 64 MiB that the library
 * declares statically, instead of the handle's own work buffers.  The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc when they apply an
 * operator: processes whose device memory is fully reserved by a pool or a budget,
 * latency-bound loops that must not block in cudaMalloc / cudaFree (cudaFree waits for
 * the whole device), or a caller applying a handle it shares with other threads.
 *   u, f   device pointers as for htlr_matvec (caller-owned, must not overlap).
 * Limits and behaviour:
 *   - operators whose scratch would exceed 64 MiB are rejected with HTLR_ENOMEM and a
 *     message giving the size needed (e.g. c2, d=3 n=32, needs about 51 MB; the
 *     n=128 operators do not fit: use htlr_matvec);
 *   - every call looks up the array's device address on the current device (an
 *     allocation-free query); the first call on a device may load the library's device
 *     code there, so make it before any CUDA stream capture;
 *   - every call on a device shares the same array: calls whose GPU work overlaps (other
 *     streams, other threads) race; nothing needs clearing between calls;
 *   - every GPU that loads the library holds the 64 MiB until the process exits.
 * Asynchronous on the handle's stream; the current device must be the handle's device.
 */
int htlr_matvec_noalloc(const htlr_handle *H, const double *u, double *f, int nrhs);

/* Options of htlr_gmres (NULL: restart 30, max_iters 3000, tol 1e-10, inner_tol 1e-6,
 * max_refine 20). */
typedef struct {
    int restart;       /* Krylov dimension m of GMRES(m), 1..200 */
    int max_iters;     /* total Arnoldi steps over all restarts (and refinements) */
    double tol;        /* target ||f - A u|| / ||f|| per right-hand side (A: the operator H) */
    double inner_tol;  /* refinement only: relative tolerance of each inner solve */
    int max_refine;    /* refinement only: maximum correction steps */
} htlr_gmres_options;

typedef struct {
    int iterations;      /* Arnoldi steps taken (all restarts and refinements) */
    int matvecs;         /* operator applications (each one covers all nrhs) */
    int refinements;     /* correction steps (0 without an inner operator) */
    double rel_residual; /* max over the right-hand sides of ||f - A u|| / ||f||, A = H */
    int converged;       /* 1 if rel_residual <= tol */
} htlr_gmres_result;

/*
 * htlr_gmres -- solve a(x) u + K u = f (the inversion of eq. (1.1); A applied by
 * HMultVec) for nrhs right-hand sides with restarted GMRES(m): FP64 Arnoldi with
 * classical Gram-Schmidt applied twice, Givens rotations, true residual at each restart.
 *   H        the operator whose residual defines convergence (FP64 or df64 for 1e-10).
 *   H_inner  NULL, or an operator of the same grid (typically mixed precision): then the
 *            solve is iterative refinement -- r = f - H u, H_inner e = r solved to
 *            inner_tol, u += e -- until ||r|| <= tol ||f||.
 *   f, u     device pointers, N x nrhs column-major; u holds the initial guess and
 *            receives the solution.
 * Allocates its Krylov workspace ((restart + 4) N nrhs doubles) for the call.
 * Synchronous.  Errors as htlr_matvec; HTLR_EINVAL for bad options.
 */
int htlr_gmres(const htlr_handle *H, const htlr_handle *H_inner, const double *f, double *u,
               int nrhs, const htlr_gmres_options *o, htlr_gmres_result *res);

/*
 * Matvec plans (no counterpart in the paper): the launch sequence of one htlr_matvec
 * (H, u, f, nrhs) captured once into a CUDA graph and replayed by one graph launch, for
 * callers that apply an operator many times to the same device buffers (iterative
 * solvers, serving loops).  u and f are fixed at creation: the caller rewrites their
 * contents between launches.  The plan borrows H (free plans before H).
 *   htlr_plan_create  captures on a private stream; errors as htlr_matvec.
 *   htlr_plan_launch  enqueues f = A u on the handle's current stream; if H's task tables
 *                     were rebuilt since the capture (htlr_autotune) it re-captures first.
 *   htlr_plan_launches  the kernel launches inside the graph (-1 for NULL).
 *   htlr_plan_free    releases the graph; NULL is a no-op.
 */
typedef struct htlr_plan htlr_plan;
int htlr_plan_create(const htlr_handle *H, const double *u, double *f, int nrhs,
                     htlr_plan **P);
int htlr_plan_launch(htlr_plan *P);
int htlr_plan_launches(const htlr_plan *P);
void htlr_plan_free(htlr_plan *P);

/* Launch shapes chosen by htlr_autotune. */
typedef struct {
    size_t task_bytes;       /* CUDA-core block stream: bytes of blocks per warp task */
    int stream_ctas_per_sm;  /* CUDA-core block stream: grid cap = 152 x this */
    int stream_threads;      /* CUDA-core block stream: threads per CTA (128 or 256) */
    int tc_stages;           /* tensor-core ring depth cap (0: the deepest that fits) */
    float ms;                /* median matvec time of the chosen shapes (ms; 0 if cached) */
    float default_ms;        /* median matvec time of the shapes the handle had before */
    int candidates;          /* configurations timed */
    int from_cache;          /* 1: taken from the process-wide table, nothing timed */
} htlr_tune_result;

/*
 * htlr_autotune -- choose the matvec's launch shapes for nrhs right-hand sides by timing
 * (no counterpart in the paper).  Coordinate descent from the handle's current shapes:
 * the stream's task size (64 KB .. 1 MB of blocks per warp task), its grid cap (2..16
 * CTAs per SM) and CTA size (128 / 256), or the tensor-core ring depth (2..4); each
 * candidate is the median of 3 matvecs (CUDA events, handle's stream) after a warm-up, on
 * scratch vectors the call allocates (2 N nrhs doubles).  Stops trying candidates when
 * the next one would exceed budget_ms of device time (0: time only the current shapes).
 * The winner is applied to H and stored in a process-wide table keyed by the operator's
 * shape (d, n, leaf, r, eta, storage, precisions, kernel, min(nrhs, RHS chunk)); a later
 * call for the same shape applies it without timing.  Results change only by rounding
 * order.  Plans captured on H re-capture on their next launch.  Synchronous.
 */
int htlr_autotune(htlr_handle *H, int nrhs, double budget_ms, htlr_tune_result *res);

/* Forget every shape htlr_autotune remembered. */
void htlr_autotune_clear_cache(void);

/* ---------------------------------------------------------------------------------
 * Serving loop (no counterpart in the paper): a request loop that keeps constructed
 * operators resident and solves a(x) u + K u = f for many concurrent requests with
 * continuous batching.  A scheduler thread owns the device: requests wait in a FIFO
 * until a slot (max_active) and HBM are free; an operator is constructed (Algorithm 1)
 * when a request first needs it and released, least recently used first, when an idle
 * one is in the way of a new one.  Each active request is a restarted GMRES(restart)
 * solve (FP64 Arnoldi with classical Gram-Schmidt twice, Givens rotations); every
 * scheduler step applies each operator once to the columns of all its requests that
 * need it (at most max_batch), so requests arriving while others iterate join the next
 * step, and converged ones leave at once.  Operators run on their own streams and their
 * steps overlap on the device.  Mixed mode: each operator has a df64 handle that defines
 * the residual and an inner handle (inner_precision) that builds the Krylov spaces, and
 * each restart is a step of iterative refinement (each inner cycle stops at inner_tol
 * times its starting residual).  A result does not depend on which requests shared its
 * batches: every column of a batched matvec and every per-request reduction is computed
 * as it would be alone.
 * --------------------------------------------------------------------------------- */
typedef struct htlr_server htlr_server;

typedef struct {
    size_t hbm_budget;    /* device bytes for resident operators, batch buffers and request
                             workspaces ((restart + 4) N doubles each); 0: 80% of free */
    int max_active;       /* requests iterating at once (slots), >= 1 */
    int max_batch;        /* columns per batched matvec, 1..64 */
    int mixed;            /* 0: FP64 operators; 1: df64 residual + inner operator */
    int inner_precision;  /* mixed: HTLR_PREC_FP32, _DF64 or _BF16X6 (far and near) */
    int restart;          /* GMRES restart length, 1..200 */
    double tol;           /* target ||f - A u|| / ||f|| (A: the FP64 or df64 operator) */
    double inner_tol;     /* mixed: relative residual reduction of each inner cycle, (0,1) */
    int max_iters;        /* Arnoldi steps per request, over all restarts */
    int use_graphs;       /* 1: batched matvecs replayed from captured plans (htlr_plan) */
    double autotune_ms;   /* > 0: htlr_autotune budget for each constructed handle */
} htlr_server_options;

typedef struct {          /* one operator of the served family (uniform grid, orth default) */
    int kernel_type;      /* htlr_kernel_type */
    double kscale, kparam;
    int d, n, leaf, r;
    double eta;
    const double *a;      /* host array of N values (natural order) or NULL (a = 0); copied */
    int storage;          /* htlr_storage: AUTO, STORED or SHARED */
} htlr_operator_spec;

enum { HTLR_REQ_QUEUED = 0, HTLR_REQ_ACTIVE = 1, HTLR_REQ_DONE = 2, HTLR_REQ_FAILED = 3 };

typedef struct {
    int status;           /* HTLR_REQ_* */
    int error;            /* HTLR_* code when failed */
    int iterations;       /* Arnoldi steps */
    int matvecs;          /* operator applications (columns of batched matvecs) */
    int refinements;      /* mixed: correction steps after the first */
    double rel_residual;  /* ||f - A u|| / ||f|| at the last residual check */
    int converged;        /* rel_residual <= tol */
    double submit_s, admit_s, done_s;  /* seconds since the server was created */
} htlr_request_info;

typedef struct {
    long long submitted, completed, failed;
    int active, pending;
    long long steps, batched_matvecs, matvec_columns;
    int max_batch_seen;
    long long constructions, evictions;
    long long bytes_in_use, bytes_peak, bytes_budget;
    int resident_operators;
} htlr_server_stats;

/* Start a server on the current device (o NULL: max_active 64, max_batch 16, mixed 1
 * with FP32 inner, restart 30, tol 1e-10, inner_tol 1e-4, max_iters 3000, graphs on,
 * no autotuning, budget 80% of free memory).  HTLR_EINVAL for bad options. */
int htlr_server_create(const htlr_server_options *o, htlr_server **S);
/* Register an operator (constructed on first use); *op_id names it in submissions. */
int htlr_server_add_operator(htlr_server *S, const htlr_operator_spec *spec, int *op_id);
/* Queue the solve of A u = f for operator op_id.  f_host (N doubles) is copied before the
 * call returns; u_host (N doubles, host) receives the solution and must stay valid until
 * the request is DONE or FAILED.  Thread-safe. */
int htlr_server_submit(htlr_server *S, int op_id, const double *f_host, double *u_host,
                       long long *req_id);
/* Current state of a request (non-blocking). */
int htlr_server_poll(htlr_server *S, long long req_id, htlr_request_info *info);
/* Block until the request is DONE or FAILED (timeout_s < 0: no limit; HTLR_ETIMEOUT). */
int htlr_server_wait(htlr_server *S, long long req_id, double timeout_s, htlr_request_info *info);
/* Counters and memory use. */
int htlr_server_get_stats(htlr_server *S, htlr_server_stats *st);
/* Finish every queued and active request, release all operators and stop the thread. */
void htlr_server_destroy(htlr_server *S);

/* Release everything the handle owns.  NULL is a no-op.  A second free of the same
 * handle is detected through a magic word and ignored (reported by htlr_last_error). */
void htlr_free(htlr_handle *H);

/* Fill *s with the structure and memory statistics. */
int htlr_info(const htlr_handle *H, htlr_stats *s);

/* Replace the stream used by later calls on H (NULL: default stream). */
int htlr_set_stream(htlr_handle *H, void *stream);

/*
 * htlr_sync -- wait for the handle's stream, then read and clear the handle's device error
 * word.  Returns HTLR_ETIMEOUT when a bounded wait of a tensor-core kernel ran out in any
 * work enqueued since the word was last read (those matvecs' results are invalid),
 * HTLR_EDEVICE for any other device-side check, HTLR_OK otherwise.  The word is cleared
 * when it is reported, so each failure is reported once and the handle stays usable.
 * The synchronous entry points (htlr_matvec_host, htlr_matvec_timed, htlr_gmres) read it
 * the same way before they return; htlr_matvec and htlr_plan_launch are asynchronous
 * and leave it to htlr_sync.
 */
int htlr_sync(const htlr_handle *H);

/*
 * htlr_set_wait_limit -- replace the handle's bounded-wait limit (htlr_options
 * tc_wait_cycles; 0 restores the default) for later matvecs.  Plans captured on H
 * re-capture on their next launch.  HTLR_EINVAL for a negative limit.
 */
int htlr_set_wait_limit(htlr_handle *H, long long cycles);

/* Message of the last failed call on this thread ("" if none). */
const char *htlr_last_error(void);

/* BF16 tensor-core FLOPs (2 M N K summed over the MMAs, padding and the six split
 * products included) one htlr_matvec of nrhs right-hand sides executes on H; 0 when H
 * has no BF16X6 block list.  Host-side count, no device work. */
double htlr_tensor_flops(const htlr_handle *H, int nrhs);

/* Device allocations (cudaMalloc) the library has made in this process so far: every
 * entry point allocates through one counted helper, so a caller can check that a call
 * (htlr_matvec_noalloc, for instance) allocated nothing. */
long long htlr_device_allocations(void);

/* Number of kernel launches the last htlr_matvec on H enqueued. */
int htlr_last_launch_count(const htlr_handle *H);

#ifdef __cplusplus
}
#endif

#endif /* HTLR_H */
