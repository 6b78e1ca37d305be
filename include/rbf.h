/*
 * rbf.h - C ABI of the B300 (sm_103a) Gaussian-RBF implicit-surface library.
 *
 * The library implements the computational core of Cuomo, Galletti, Giunta,
 * Starace, "Surface Reconstruction from Scattered Point via RBF Interpolation on
 * GPU" (Algorithm 1, steps 1-3):
 *   step 1  extend the cloud X with off-surface points X+ and X- (Sec. II.A.1)
 *   step 2  find the interpolant: solve A c = b (Eq. RBFsys) with the Gaussian
 *           entries of Eq. matrixEntries, truncated at a cut-off so that the
 *           product A z is local (Sec. III.A), by GMRES with a restricted
 *           additive Schwarz preconditioner (Sec. III.A), matrix-free
 *           ("MatShell", Sec. III.B)
 *   step 3  evaluate P_f on a grid (Eq. matxvet; Algorithm 3 is the paper's
 *           evaluation kernel)
 *
 * Conventions (fixed for every entry point):
 *   - Kernel.  phi(r) = exp(-r^2 / (2 sigma^2)).  The paper's factor
 *     1/(sqrt(2 pi) sigma) (Table I, Eq. matrixEntries) is left out: it
 *     multiplies every weight by the same constant and leaves P_f unchanged.
 *   - Truncation.  With cut-off factor k > 0 the operator keeps the pairs with
 *     |c_i - c_j| < k sigma (strict); every dropped entry is below exp(-k^2/2).
 *     (For k >= 5.77 the tensor-core product also keeps some pairs just beyond
 *     the radius, whose entries are below 2^-24: see rbf_matvec.)
 *     k = 0 means untruncated (dense).  0 <= k <= 12.
 *   - Centres.  float4 per centre (x, y, z, unused), 16-byte aligned, in the
 *     order [X; X+; X-] that rbf_build_centers writes (Sec. II.A.1).
 *   - Memory.  Every array argument is DEVICE memory owned by the caller unless
 *     a comment says "host".  The library never frees or retains a caller
 *     pointer beyond the call, except that a plan keeps its own copies of the
 *     centres it was built from.
 *   - Streams.  `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream.  Work is enqueued on it; calls that return host values
 *     (reports, counts, info) synchronise that stream before returning.
 *   - Errors.  Functions return rbf_status and never abort or print.  A
 *     human-readable reason for the last failure on a context is returned by
 *     rbf_last_error.  On error, outputs are unspecified.
 *   - Threads.  A context and the plans made from it may be used by one host
 *     thread at a time.
 */
#ifndef RBF_H
#define RBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RBF_VERSION 1

typedef enum {
    RBF_OK = 0,
    RBF_ERR_INVALID = 1,        /* bad argument: null pointer, size, sigma <= 0, k out of range, non-finite */
    RBF_ERR_OOM = 2,            /* a device allocation failed */
    RBF_ERR_CUDA = 3,           /* a CUDA runtime call or kernel launch failed */
    RBF_ERR_NOT_CONVERGED = 4,  /* solver stopped at its iteration cap above tolerance (weights still valid) */
    RBF_ERR_BREAKDOWN = 5,      /* Arnoldi produced a non-finite value */
    RBF_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired (reported by the next call on the
                                   context that launches a product or synchronises) */
    RBF_ERR_NOT_SPD = 7,        /* a block factorisation failed even after the shift escalation */
    RBF_ERR_UNSUPPORTED = 8,    /* configuration outside the implemented range (message says which) */
    RBF_ERR_RANGE = 9           /* a device-side value left a documented range (message says which);
                                   reported like RBF_ERR_TIMEOUT, results of that launch invalid */
} rbf_status;

typedef struct rbf_ctx rbf_ctx;
typedef struct rbf_plan rbf_plan;

/* Library version (RBF_VERSION of the build). */
int rbf_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all contexts and threads).  Host-only, no device work. */
int64_t rbf_launch_count(void);

/* Static string naming a status code. */
const char *rbf_status_string(rbf_status s);

/* Create a context on CUDA device `device` (made current for every call on the
 * context).  *ctx receives a host-owned handle; destroy it with rbf_ctx_destroy,
 * after the plans, batches and networks made on it (their destroy functions do
 * not touch the context; every other call on them does).  The first context on
 * a device also loads the allocation-free product's code and its 4 MiB scratch
 * array (see rbf_matvec_dense_noalloc), which stay until the process exits. */
rbf_status rbf_ctx_create(rbf_ctx **ctx, int device);
rbf_status rbf_ctx_destroy(rbf_ctx *ctx);

/* Reason for the last failure on this context (empty string if none).  The
 * pointer stays valid until the next call on the context. */
const char *rbf_last_error(const rbf_ctx *ctx);

/* ------------------------------------------------------------------------
 * Step 1 (Sec. II.A.1-2): extended data set.
 *   pts, nrm : N x 3 float, row-major (x, y, z per point); normals oriented
 *              outward and of unit length (used as given).
 *   delta    : offset along the normal; delta <= 0 selects 1% of the diagonal of
 *              the bounding box of pts (the paper's default, Sec. II.A.1).
 *   target   : value assigned on X+ (and -target on X-); target <= 0 selects
 *              `delta` (signed-distance targets).  The paper's +-1 is target = 1.
 *   centers  : out, 3N float4 (x, y, z, 0): [X; X + delta n; X - delta n].
 *   targets  : out, 3N float: [0...; +target...; -target...].
 *   delta_out: host, optional (may be NULL): the delta used.
 * Errors: RBF_ERR_INVALID for N <= 0, null or misaligned pointers, or a
 * non-finite coordinate (checked on the device; one stream synchronisation). */
rbf_status rbf_build_centers(rbf_ctx *ctx, const float *pts, const float *nrm, int64_t N,
                             float delta, float target, float *centers, float *targets,
                             float *delta_out, void *stream);

/* ------------------------------------------------------------------------
 * Plan: the matrix-free operator A~ over a fixed set of centres (the paper's
 * MatShell, Sec. III.B), i.e. cell binning (Sec. III.A "truncation area",
 * Algorithm 2) plus the block/tile structure the kernels walk.
 *
 * Binning is a definition shared with the tests:
 *   lo = componentwise minimum of the centres, ext = hi - lo (float32);
 *   cell edge hc = cell_edge when cell_edge > 0; otherwise k sigma /
 *   cells_per_cutoff (k > 0, the truncation area of Algorithm 2), or the
 *   layout choice max(min(max(ext)/8, 3 sigma), max(ext)/128) in double (k = 0,
 *   Gaussian), max(ext)/8 (k = 0, inverse multiquadric); 1 if ext is 0;
 *   fine cells hf = hc / 2^levels; inv = (float)(2^levels / hc) computed in
 *   double; q_d = floor((c_d - lo_d) * inv) in float32;
 *   key = Morton interleave (x in bit 0) of q; cell = key >> (3 levels);
 *   centres are ordered by a stable sort on key.  At most 1024 fine cells per
 *   axis (RBF_ERR_UNSUPPORTED otherwise).  Any positive cell edge gives the
 *   same operator: the kernels enumerate every cell within the cut-off.
 * After the sort, the centres of each cell are reordered among themselves
 * (an internal layout, not part of the definition): runs of at most 4096
 * consecutive positions counted from the cell start are split recursively at
 * a median along the axis of largest extent, so that the runs of 32 (source
 * blocks) and of 128 (target tiles) counted from the cell start are subtrees:
 * any two such runs of one 4096-run are separated along some axis (the
 * largest coordinate of one is <= the smallest of the other).
 * ------------------------------------------------------------------------ */
typedef struct {
    float sigma;            /* Gaussian width, > 0 */
    float k;                /* cut-off factor: pairs with |d| < k sigma; 0 = untruncated */
    int cells_per_cutoff;   /* s in hc = k sigma / s; 0 selects 1 */
    int levels;             /* fine levels per cell (0..7); -1 selects 3 */
    int product;            /* kernel of the float32 product and grid evaluation: RBF_PRODUCT_TC (0) or
                               RBF_PRODUCT_SIMT (1); both compute the same sum (see rbf_matvec) */
    int kernel;             /* radial function: RBF_KERNEL_GAUSSIAN (0, the paper's choice) or
                               RBF_KERNEL_IMQ (1), see below */
    float beta;             /* RBF_KERNEL_IMQ: exponent, 0 < beta <= 16 */
    float cell_edge;        /* cell edge hc of the binning; 0 selects the default rule above; finite, >= 0 */
} rbf_plan_params;

/* Radial functions (Table I).  The Gaussian exp(-r^2 / (2 sigma^2)) is the
 * method's; the inverse multiquadric (1 + r^2 / sigma^2)^(-beta) is Table I's
 * (1 + r^2)^(-beta) with the length scale sigma (positive definite for every
 * beta > 0).  IMQ plans: the products and the grid evaluation run a direct
 * float32 kernel (one thread per target; the `product` choice does not apply),
 * true residuals are native float64 whatever the residual mode, k > 0 truncates
 * at k sigma with entry error (1 + k^2)^(-beta) (large: IMQ decays
 * algebraically), k = 0 keeps every pair; the learned preconditioner and the
 * batched solve take Gaussian plans only (RBF_ERR_UNSUPPORTED). */
enum { RBF_KERNEL_GAUSSIAN = 0, RBF_KERNEL_IMQ = 1 };

enum {
    RBF_PRODUCT_TC = 0,     /* exponents -|u - v|^2 of a 128 x 32 tile by tcgen05.mma (tf32 head + tail
                               split, ~22 bits), exp2 and the sum on the CUDA cores */
    RBF_PRODUCT_SIMT = 1    /* everything on the CUDA cores (packed float32 FMA) */
};

typedef struct {
    int64_t n;              /* centres */
    int64_t ncells;         /* entries of the dense cell table (2^(3(nbits-levels))) */
    int64_t nblocks;        /* source blocks (runs of <= 32 centres inside one cell) */
    int64_t nchunks;        /* target tiles (runs of <= 128 consecutive binned centres of one cell) */
    int64_t pairlist_len;   /* (tile, block) entries that survive the box test */
    int64_t nsegments;      /* work items of the product kernels */
    int nbits;              /* Morton bits per axis */
    int levels;
    float lo[3];
    float inv;              /* fine cells per unit length (float32) */
    float sigma, k;
    double cell_edge;       /* the cell edge hc used (double, before inv is rounded) */
    int symmetric;          /* 1: the tensor-core product evaluates each in-range pair once and adds
                               its transposed share to the source's row (plans whose (tile, block)
                               list averages fewer than 128 entries per tile); 0: from both sides */
} rbf_plan_info;

/* Build a plan over n centres (device float4 array, caller order).  The plan
 * copies what it needs; `centers` may be freed after the call returns.
 * Synchronises `stream` once (to size the cell table).
 * Errors: RBF_ERR_INVALID (n <= 0, sigma <= 0 or non-finite, k < 0 or > 12,
 * non-finite centre), RBF_ERR_UNSUPPORTED (domain too large for the cell grid),
 * RBF_ERR_OOM, RBF_ERR_CUDA. */
rbf_status rbf_plan_create(rbf_ctx *ctx, const float *centers, int64_t n, const rbf_plan_params *p,
                           rbf_plan **plan, void *stream);
rbf_status rbf_plan_destroy(rbf_plan *plan);

/* Host-side summary of the plan (no device work). */
rbf_status rbf_plan_get_info(const rbf_plan *plan, rbf_plan_info *info);

/* Copy the binning out (device pointers, any may be NULL):
 *   perm       : n int32, perm[p] = caller index of the centre at binned position p
 *   keys       : n uint32, Morton key of binned position p (sorted by cell; the
 *                order inside a cell is the layout described above)
 *   cell_start : ncells int32, first binned position of each cell code
 *   cell_end   : ncells int32, one past the last (start == end == 0 when empty) */
rbf_status rbf_plan_export_binning(rbf_plan *plan, int32_t *perm, uint32_t *keys, int32_t *cell_start,
                                   int32_t *cell_end, void *stream);

/* ------------------------------------------------------------------------
 * The truncated product y = A~ z (Sec. III.A, Eq. matrixEntries), float32
 * arithmetic with exp2 on the special-function unit, caller order.
 *   z, y : n float each (may not alias).
 * Per-pair error: relative ~1e-6 of the term.  Cut-off: the CUDA-core product
 * (RBF_PRODUCT_SIMT) tests every pair in float32 (it can differ from an exact
 * test only within rounding of the radius).  The tensor-core product
 * (RBF_PRODUCT_TC) tests them too when exp(-k^2/2) >= 2^-24 (k < 5.77); for
 * k >= 5.77 it sums every pair of each (32-target quarter, 32-source block)
 * combination that the plan could not exclude, so besides every pair within
 * k sigma it includes pairs of straddling combinations just beyond it, each of
 * entry below exp(-k^2/2) < 2^-24 - below float32's resolution of the unit
 * diagonal and below the truncation bound itself.  The pair counts, the
 * residuals and the assembled matrix use the strict cut-off. */
rbf_status rbf_matvec(rbf_plan *plan, const float *z, float *y, void *stream);

/* Number of algorithmic pairs (i, j) with |c_i - c_j| < k sigma, i = j included
 * (all n^2 when k = 0), decided in double precision.  `count` is host memory.
 * Costs about one double-precision product. */
rbf_status rbf_count_pairs(rbf_plan *plan, int64_t *count, void *stream);

/* Number of (target, source) pairs the tensor-core product evaluates: for every
 * pair-list entry, each quarter of 32 targets of its tile whose box test does not
 * exclude the block, times the block's sources (pairs beyond the cut-off inside
 * such quarter-block combinations are evaluated and kept, see rbf_matvec).  Divided by
 * rbf_count_pairs it is the product's waste ratio (>= 1; n^2 / n^2 = 1 when every
 * pair is kept).  `count` is host memory; synchronises `stream`. */
rbf_status rbf_count_candidate_pairs(rbf_plan *plan, int64_t *count, void *stream);

/* True residual r = b - A~ x with float64-class accuracy, caller order.
 *   mode  : RBF_RESIDUAL_DF (default, 0): double-float arithmetic (pairs of
 *           float32 with error-free transformations, table-driven exp2) on the
 *           float32 pipes, per-term relative error ~1e-14;
 *           RBF_RESIDUAL_F64 (1): native float64 difference, square distance,
 *           exp and accumulation (B300's FP64 rate makes this ~25x slower).
 *           The cut-off is decided on the float64-class squared distance.
 *   b : n float (targets), x : n double, r : n double (out).
 *   norms : host, optional, [|r|_2, |b|_2]. */
enum { RBF_RESIDUAL_DF = 0, RBF_RESIDUAL_F64 = 1 };
rbf_status rbf_residual(rbf_plan *plan, const float *b, const double *x, double *r, double *norms, int mode,
                        void *stream);

/* ------------------------------------------------------------------------
 * Assembled truncated matrix (Algorithm 2, Sec. III.B): the matrix of the
 * plan built entry by entry and kept as CSR, for comparison with the
 * matrix-free product.  The plan owns it until rbf_plan_release_csr or
 * rbf_plan_destroy.
 *
 * Layout (device, binned order: row p and column c are binned positions; the
 * caller index of position p is perm[p] from rbf_plan_export_binning):
 *   row_ptr : n + 1 int64, row p is entries [row_ptr[p], row_ptr[p+1]);
 *             every row_ptr[p] is a multiple of 4 (rows are padded)
 *   col     : stored int32 column positions
 *   val     : stored float32 values
 * Entries: every pair with |c_i - c_j| < k sigma (decided as rbf_count_pairs
 * decides, so nnz equals that count); for an untruncated plan (k = 0), every
 * pair closer than 13 sigma (the others are below 2.2e-37).  Values
 * exp(-|c_i - c_j|^2 / (2 sigma^2)) = 2^-t in float32, from the float32 squared
 * distance (relative error of t below 7 x 2^-24) through ex2.approx: relative
 * error below 2^-21 + 7 x 2^-24 ln(2) t; no 1/(sqrt(2 pi) sigma) prefactor.  Columns of a row are grouped by
 * source block (ascending inside a block), not sorted.  Padding entries have
 * the row's own position as column and value 0; a row holds each real column
 * once.
 *
 * rbf_plan_assemble: builds the matrix, replacing a previous one.  nnz, stored
 * (host, both required): entries within the cut-off and with the padding; set
 * even when the call fails for size.  max_bytes > 0 caps the matrix's size
 * (8 (stored + n + 1) bytes); RBF_ERR_OOM when that cap, or the device's free
 * memory less 2 GiB, is exceeded (then nothing is kept).  Synchronises `stream`.
 * Errors: RBF_ERR_INVALID (null pointers), RBF_ERR_OOM, RBF_ERR_CUDA. */
rbf_status rbf_plan_assemble(rbf_plan *plan, int64_t max_bytes, int64_t *nnz, int64_t *stored, void *stream);
/* Free the assembled matrix (no-op without one). */
rbf_status rbf_plan_release_csr(rbf_plan *plan);
/* Copy the assembled matrix out: row_ptr n + 1 int64, col `stored` int32, val
 * `stored` float (device; any may be NULL).  RBF_ERR_INVALID without a matrix. */
rbf_status rbf_plan_export_csr(rbf_plan *plan, int64_t *row_ptr, int32_t *col, float *val, void *stream);
/* y = A~ z through the assembled matrix (float32, caller order; z and y n
 * floats, distinct).  RBF_ERR_INVALID without a matrix. */
rbf_status rbf_spmv(rbf_plan *plan, const float *z, float *y, void *stream);

/* ------------------------------------------------------------------------
 * Restricted additive Schwarz preconditioner (Sec. III.A, RASM).
 * Subdomains are defined on the binned order: cores are consecutive runs of
 * `core` positions; subdomain i is the run of exactly min(block, n) positions
 * starting at clamp(s_i - (block - core)/2, 0, n - block), s_i = i*core.  A_i is
 * the untruncated Gaussian matrix of subdomain i, factorised in float32 as
 * A_i + shift*I = L_i L_i^T.  With restricted = 1 the apply writes only the core
 * entries of each local solve (RASM); with restricted = 0 it adds whole local
 * solves (additive Schwarz, float atomics: not bitwise reproducible).
 * ------------------------------------------------------------------------ */
typedef struct {
    int core;               /* positions per core, 1 <= core <= block */
    int block;              /* subdomain size, 1 <= block <= 128 */
    float shift;            /* diagonal shift (absolute; diag(A) = 1), >= 0 */
    int restricted;         /* 1 = RASM (default), 0 = additive */
    int escalate;           /* if non-zero, a failed block retries with shift*10 up to 4 times */
} rbf_schwarz_params;

/* Assemble and factorise all blocks.  `failed` (host, optional) receives the
 * number of blocks whose factorisation still failed; such blocks act as the
 * identity.  Returns RBF_ERR_NOT_SPD if failed > 0 (the preconditioner is still
 * usable). */
rbf_status rbf_schwarz_setup(rbf_plan *plan, const rbf_schwarz_params *p, int64_t *failed, void *stream);

/* z = M^-1 v with the factorised blocks, caller order, float in and out. */
rbf_status rbf_schwarz_apply(rbf_plan *plan, const float *v, float *z, void *stream);

/* ------------------------------------------------------------------------
 * Step 2: flexible GMRES(m) with right preconditioning (Sec. III.A: GMRES with
 * RASM).  Precision: product and preconditioner in float32; Arnoldi basis,
 * classical Gram-Schmidt applied twice, Hessenberg least squares and the
 * solution vector in float64.  Each restart recomputes the true residual with
 * rbf_residual's float64-accurate kernel (iterative refinement:
 * x += GMRES(b - A~ x)).
 * ------------------------------------------------------------------------ */
enum { RBF_PRECOND_NONE = 0, RBF_PRECOND_SCHWARZ = 1, RBF_PRECOND_MLP = 2 };

typedef struct rbf_mlp rbf_mlp;   /* learned block preconditioner, see below */

typedef struct {
    int m;                  /* restart length, 1..512 (default 50 when 0) */
    int max_it;             /* cap on inner iterations in total (default 500 when 0) */
    double tol;             /* stop when |b - A~ x|_2 <= tol |b|_2 (default 1e-6 when 0) */
    int precond;            /* RBF_PRECOND_* */
    rbf_schwarz_params schwarz;
    int fixed_iterations;   /* non-zero: run exactly max_it iterations, ignoring tol */
    int true_residual_each_restart; /* non-zero (default): float64 residual at every restart;
                                       zero: float32 product at restarts, float64 residual at the end */
    int residual_mode;      /* RBF_RESIDUAL_DF (0) or RBF_RESIDUAL_F64 (1), see rbf_residual */
    rbf_mlp *mlp;           /* RBF_PRECOND_MLP: the trained network */
    float mlp_lambda;       /* RBF_PRECOND_MLP: the shift the network was trained for */
    int mlp_initial_guess;  /* RBF_PRECOND_MLP: start from x0 = a network(b) instead of 0, with
                               a = <b, A~ g> / <A~ g, A~ g> for g = network(b) (one more product):
                               the scaling that minimises the starting residual, so that a poor
                               guess is shrunk (or dropped, a = 0) instead of starting the solve
                               above |b| */
    int assembled;          /* non-zero: the float32 products use the plan's assembled matrix
                               (rbf_plan_assemble; RBF_ERR_INVALID without one); the float64
                               true residuals stay matrix-free */
} rbf_solve_params;

typedef struct {
    int iterations;         /* inner iterations (products) performed */
    int restarts;           /* completed cycles */
    int converged;          /* 1 if the true residual met tol */
    int precond_failed_blocks;
    double residual_estimate;   /* last |g_{j+1}| / |b| from the Givens recursion */
    double residual_true;       /* final |b - A~ x| / |b| in float64 */
    double ms_setup;            /* preconditioner set-up, milliseconds (CUDA events) */
    double ms_solve;            /* iterations incl. true residuals, milliseconds */
    int64_t matvec_pairs;       /* float32 product pair evaluations (algorithmic pairs x products),
                                   0 if the plan has not counted its pairs */
    int matvec_launches;        /* float32 products inside the solve */
    int residual_launches;      /* float64 true-residual products inside the solve */
    double ms_matvec;           /* summed CUDA-event time of the float32 products */
    double ms_residual;         /* summed CUDA-event time of the float64 residual products */
    double ms_precond;          /* summed CUDA-event time of the preconditioner applications */
    double guess_scale;         /* mlp_initial_guess: the factor a applied to the network's guess g
                                   (a minimises |b - a A~ g|; 0 when the guess was not used) */
    double guess_residual;      /* mlp_initial_guess: |b - a A~ g| / |b| with the float32 product
                                   (at most 1: the guess never starts above x0 = 0) */
} rbf_report;

/* Solve A~ x = b on a plan.  b: n float (caller order); x: n double (out,
 * caller order).  `report` (host) may be NULL.  Returns RBF_ERR_NOT_CONVERGED
 * when the cap is reached above tol (x holds the last iterate; with
 * fixed_iterations this is RBF_OK). */
rbf_status rbf_plan_solve(rbf_plan *plan, const float *b, const rbf_solve_params *p, double *x,
                          rbf_report *report, void *stream);

/* One-shot form of the paper's step 2: builds a plan, solves, frees the plan. */
rbf_status rbf_solve(rbf_ctx *ctx, const float *centers, const float *targets, int64_t n,
                     const rbf_plan_params *pp, const rbf_solve_params *sp, double *weights,
                     rbf_report *report, void *stream);

/* ------------------------------------------------------------------------
 * Density measures of the cloud (Sec. IV), for choosing sigma: nearest-neighbour
 * distances, the separation distance (Eq. sepDist), h_max, and the fill
 * distance (Eq. fillDist) over caller-given probe points of the domain Omega,
 * with the paper's sigma rules.
 * ------------------------------------------------------------------------ */
typedef struct {
    double q;            /* separation distance 1/2 min_{i!=j} |x_i - x_j| (0 with duplicate points) */
    double h_max;        /* max_j min_{i!=j} |x_i - x_j| */
    double mean_nn;      /* mean nearest-neighbour distance */
    double fill;         /* max over the probes of the distance to the nearest point; NaN without probes */
    double sigma_q;      /* 2 q (Eq. h1) */
    double sigma_fill;   /* fill sqrt(2) (Eq. h2) */
    double sigma_hmax;   /* h_max sqrt(2), the fill distance estimate of Eq. hmax */
    float cell;          /* cell edge the search used */
} rbf_density;

/* points: n float4 (x, y, z, unused), probes: m float4 or NULL (m = 0), device,
 * 16-byte aligned; cell: search cell edge, <= 0 chooses one; nn: NULL or n
 * floats receiving each point's nearest-neighbour distance (caller order).
 * Distances are float32 (exact nearest neighbour, float32 arithmetic).
 * Synchronises `stream`.  Errors: RBF_ERR_INVALID (n < 2, non-finite
 * coordinates, null or misaligned pointers), RBF_ERR_UNSUPPORTED (extent too
 * large for the binning), RBF_ERR_OOM, RBF_ERR_CUDA. */
rbf_status rbf_density_measures(rbf_ctx *ctx, const float *points, int64_t n, const float *probes, int64_t m,
                                float cell, float *nn, rbf_density *out, void *stream);

/* ------------------------------------------------------------------------
 * Step 3 (Eq. matxvet): P_f at the nodes of a structured grid,
 * xi = lo + i (hi - lo)/(dims - 1) per axis (dims = 1 puts the node at lo),
 * written x fastest: f[(iz * dims[1] + iy) * dims[0] + ix].  The sum uses the
 * plan's cut-off (k sigma, or untruncated when k = 0); float32 arithmetic.
 * ------------------------------------------------------------------------ */
typedef struct {
    float lo[3];
    float hi[3];
    int64_t dims[3];        /* each >= 1; product < 2^31 */
} rbf_grid;

/* weights: n double (caller order); f: dims product float (out). */
rbf_status rbf_plan_eval_grid(rbf_plan *plan, const double *weights, const rbf_grid *g, float *f,
                              void *stream);

/* Number of (node, centre) pairs within the cut-off for this grid (nodes x n
 * when k = 0), decided in double precision on the float32 node coordinates the
 * evaluation uses.  `count` is host memory. */
rbf_status rbf_count_grid_pairs(rbf_plan *plan, const rbf_grid *g, int64_t *count, void *stream);

/* Number of (node slot, centre) pairs the grid evaluation evaluates, counted like
 * rbf_count_candidate_pairs over the grid's bricks (128 node slots each, cut into
 * quarters of 32; the bricks and quarters are powers of two along each axis, chosen
 * from the grid's spacings so that their boxes are compact; slots past the grid's
 * edge are counted).  Divided by rbf_count_grid_pairs it is the grid evaluation's
 * waste ratio.  `count` is host memory; synchronises `stream`. */
rbf_status rbf_count_grid_candidate_pairs(rbf_plan *plan, const rbf_grid *g, int64_t *count, void *stream);

/* One-shot form: plan from (centers, n, pp), evaluate, free. */
rbf_status rbf_eval_grid(rbf_ctx *ctx, const float *centers, const double *weights, int64_t n,
                         const rbf_plan_params *pp, const rbf_grid *g, float *f, void *stream);

/* ------------------------------------------------------------------------
 * Step 4 of Algorithm 1 without the rendering: the level set {f = iso} of a grid
 * field (as written by rbf_eval_grid) as a triangle buffer.  Marching tetrahedra
 * over the six tetrahedra of each cell around its (0,0,0)-(1,1,1) diagonal;
 * a node is inside when f < iso; an edge point is interpolated linearly from the
 * edge's node of smaller index; each triangle (v0, v1, v2) has its normal
 * (v1 - v0) x (v2 - v0) pointing from inside to outside; cells with a NaN node
 * give none.  Triangles come in cell order (x fastest), then tetrahedron, then
 * triangle.  With data points and band > 0 only cells whose centre lies within
 * band of a data point contribute (the surrounding volume M_ext^eps of Sec.
 * II.A.3; points = the cloud X, float4, device, 16-byte aligned).
 *   f         : device float, dims[0] x dims[1] x dims[2], x fastest; dims >= 2
 *   triangles : device float, 9 per triangle (x, y, z of v0, v1, v2), or NULL to
 *               count only; capacity = triangles it can hold
 *   ntri      : host, the number of triangles of the level set
 * Synchronises `stream`.  Errors: RBF_ERR_INVALID (bad grid, non-finite iso,
 * capacity below the count), RBF_ERR_OOM, RBF_ERR_CUDA. */
rbf_status rbf_isosurface(rbf_ctx *ctx, const float *f, const rbf_grid *g, float iso, const float *points,
                          int64_t npoints, float band, float *triangles, int64_t capacity, int64_t *ntri,
                          void *stream);

/* ------------------------------------------------------------------------
 * Learned block preconditioner (not in the paper: it stands in for the exact
 * subdomain solve of the restricted additive Schwarz method, Sec. III.A).
 * Blocks are the Schwarz subdomains of 64 centres without overlap.  Input of a
 * block and vector r (256 values): the 64 offsets (c_k - c_mean)/sigma, x y z per
 * centre, then rho = 8 r_k / |r|_2 (unit mean square).  Network
 * 256 -> 256 -> 256 -> 64, ReLU, plus a skip connection adding rho to the output;
 * weights W[out][in] row-major followed by the bias, layer by layer
 * (RBF_MLP_NPARAMS floats: W1 256x256, b1, W2 256x256, b2, W3 64x256, b3);
 * inference uses a BF16 copy of the weights with FP32 accumulation.  The output
 * approximates 8 lambda (A_i + lambda I)^-1 r / |r|; the preconditioner writes
 * output * |r| / (8 lambda) on the block.  Blocks whose output is not finite fall
 * back to the exact Schwarz block solve (set up automatically with block 64,
 * core 64, shift lambda) and are counted in rbf_report.precond_failed_blocks.
 * ------------------------------------------------------------------------ */
#define RBF_MLP_NPARAMS 148032
#define RBF_MLP_IN 256
#define RBF_MLP_OUT 64

typedef struct {
    int epochs;             /* passes over the data */
    int batch;              /* rows per Adam step (consecutive rows, no shuffling) */
    float lr;               /* Adam step size (beta1 0.9, beta2 0.999, eps 1e-8) */
} rbf_train_params;

/* host_params: RBF_MLP_NPARAMS floats (host), the initial weights. */
rbf_status rbf_mlp_create(rbf_ctx *ctx, const float *host_params, rbf_mlp **mlp);
rbf_status rbf_mlp_destroy(rbf_mlp *mlp);
/* Copy the FP32 master weights to host memory (RBF_MLP_NPARAMS floats). */
rbf_status rbf_mlp_get_params(rbf_mlp *mlp, float *host_params);

/* Training data from a plan: for sample s with subdomain block_ids[s] (64-centre
 * blocks without overlap, device int32) and right-hand side R[s] (device, 64
 * float, caller-drawn random numbers): X[s] (256 float, out) and
 * Y[s] = 8 lambda (A_i + lambda I)^-1 R[s] / |R[s]| (64 float, out) from an exact
 * float64 Cholesky solve.  failed (host, optional): samples whose factorisation
 * failed. */
rbf_status rbf_mlp_make_data(rbf_plan *plan, float lambda, const int32_t *block_ids, const float *R, int64_t ns,
                             float *X, float *Y, int64_t *failed, void *stream);

/* Y = network(X) for `rows` inputs (device); use_bf16 selects the inference weights. */
rbf_status rbf_mlp_forward(rbf_mlp *mlp, const float *X, int64_t rows, float *Y, int use_bf16, void *stream);

/* Mean squared error of the FP32-weight network on (X, T) and, if host_grad is
 * not NULL, its gradient with respect to the master weights (host,
 * RBF_MLP_NPARAMS floats, same layout).  rows <= 65536. */
rbf_status rbf_mlp_loss_grad(rbf_mlp *mlp, const float *X, const float *T, int64_t rows, double *loss,
                             float *host_grad, void *stream);

/* Adam training on (X, T) (device, ns rows); loss_history (host, epochs doubles,
 * optional) receives the mean loss of every epoch. */
rbf_status rbf_mlp_train(rbf_mlp *mlp, const float *X, const float *T, int64_t ns, const rbf_train_params *p,
                         double *loss_history, void *stream);

/* ------------------------------------------------------------------------
 * Batched solve of many independent problems (for example many clouds of
 * uneven size, each with its own sigma): one plan per problem, solved together
 * by flexible GMRES in lockstep with every step on the device, so that a whole
 * solve is a single CUDA graph launch.  The product runs one CTA per
 * (problem, segment) work item, longest first: the tensor-core kernel when every
 * plan takes RBF_PRODUCT_TC, else a persistent CUDA-core kernel whose CTAs take
 * items from an atomic counter; the Arnoldi reductions are segmented per problem; the Givens
 * rotations and the triangular solve run on the device.  The captured solve has
 * max_it steps (restarted every m <= 64, each restart with a float64-class true
 * residual); with p->fixed_iterations every problem takes all of them, as in the
 * paper's timing protocol (Table II); otherwise a problem stops at p->tol (its
 * residual estimate within a cycle, its true residual at a restart) and the
 * kernels skip its work from then on.  Each problem reports its own true
 * residual and its iteration count.
 * ------------------------------------------------------------------------ */
typedef struct rbf_batch rbf_batch;

typedef struct {
    double ms_setup;            /* preconditioner set-up and buffers, milliseconds */
    double ms_solve;            /* gather, graph launch, scatter, milliseconds (CUDA events) */
    int64_t graph_nodes;        /* nodes of the captured solve (0 when it was replayed) */
    int recaptured;             /* 1 if this call captured the graph */
    int persistent_ctas;        /* CTAs of the persistent CUDA-core product (unused by the tensor-core one) */
    int64_t work_items;         /* (problem, segment) items per product */
    int converged;              /* problems whose true residual met tol */
    double worst_residual;      /* largest relative true residual over the problems */
    int precond_failed_blocks;
} rbf_batch_stats;

/* Group `nplans` plans (made on `ctx`, kept alive by the caller until the batch
 * is destroyed) into a batch.  Re-cuts the plans' pair lists into segments of a
 * common length for the persistent product (the plans stay usable). */
rbf_status rbf_batch_create(rbf_ctx *ctx, rbf_plan *const *plans, int nplans, rbf_batch **batch, void *stream);
rbf_status rbf_batch_destroy(rbf_batch *batch);

/* Total number of centres (sum over the plans). */
int64_t rbf_batch_size(const rbf_batch *batch);

/* y = A~ z for every problem; z, y: concatenations of the problems' vectors in
 * plan order (caller order within each problem), float. */
rbf_status rbf_batch_matvec(rbf_batch *batch, const float *z, float *y, void *stream);

/* Solve every problem: b (float) and x (double, out) are concatenations as above;
 * p->fixed_iterations: every problem takes max_it steps, else each stops at
 * p->tol (1e-6 if <= 0); p->m <= 64; p->precond NONE or SCHWARZ (the
 * Schwarz set-up runs on every plan when its block size changes).  reports: host
 * array of nplans (may be NULL); stats: host (may be NULL). */
rbf_status rbf_batch_solve(rbf_batch *batch, const float *b, const rbf_solve_params *p, double *x,
                           rbf_report *reports, rbf_batch_stats *stats, void *stream);

/* Choose the Schwarz subdomain size: for each candidate block size (block
 * Jacobi: core = block, the shift of p) run a short solve (min(m, 20)
 * iterations) of b and score it by decades of worst-case residual reduction per
 * millisecond.  *best receives the winner; scores (host, ncand, may be NULL)
 * the scores.  The batch keeps a Schwarz set-up between solves while core,
 * block, shift, restricted and escalate are unchanged. */
rbf_status rbf_batch_autotune(rbf_batch *batch, const float *b, const rbf_solve_params *p, const int *candidates,
                              int ncand, int *best, double *scores, void *stream);

/* ------------------------------------------------------------------------
 * Allocation-free untruncated product (the paper has no counterpart: it is a
 * service to callers of this library that cannot allocate device memory when
 * they call in, for example a host that reserves its whole device-memory
 * budget at start-up and forbids later allocation, or code running inside
 * another framework's memory pool or a real-time loop).
 *
 * y = A z with A_ij = exp(-|c_i - c_j|^2 / (2 sigma^2)) over all pairs (no
 * cut-off, no plan, no binning), float32 arithmetic, caller order; the same
 * operator as rbf_matvec on a plan with k = 0.
 *   centers : n float4 (x, y, z, unused), 16-byte aligned; z, y : n float,
 *             distinct.  All device memory owned by the caller.
 *   n       : 1 <= n <= 32768; larger n returns RBF_ERR_UNSUPPORTED with the
 *             limit in rbf_last_error.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  Its scratch is a 4 MiB file-scope device array (32 x 32768 float
 * partial sums) that every GPU loading the library holds until the process
 * exits.  It is allocated when the module holding it loads, which
 * rbf_ctx_create forces (it also resolves the array's device address with
 * cudaGetSymbolAddress, with the context's device current, and loads the two
 * kernels), so the device memory is taken then and never by a call; create
 * the context before any stream capture.  All calls share the array and it keeps the last call's
 * contents; every entry a call reads is written earlier in the same call, so
 * nothing needs clearing, but calls whose work overlaps on the GPU (different
 * streams, or different host threads) race on it and must be serialised by the
 * caller. */
rbf_status rbf_matvec_dense_noalloc(rbf_ctx *ctx, const float *centers, int64_t n, float sigma, const float *z,
                                    float *y, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RBF_H */
