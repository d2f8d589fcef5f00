/*
 * ifmm.h -- C ABI of the GB300 (sm_103a) Inverse Fast Multipole Method library.
 *
 * The method is that of Ambikasaran & Darve, "The Inverse Fast Multipole Method: an O(N)
 * fast direct solver" (arXiv:1407.1572): a dense N x N FMM matrix A~ is written exactly as an
 * extended sparse system in the particles x, multipoles y and locals z of every box of a
 * uniform quadtree (Section 4.1), and that system is eliminated level by level, box by box
 * (Algorithm 1); fill-in between well-separated boxes is compressed into the box bases on the
 * fly, fill-in between neighbours stays dense. Back substitution runs the levels downward in
 * the reverse order (Algorithm 2). The problem statement the calls follow is that of
 * Section 1: given b and a tolerance eps, solve A x = b for an FMM matrix A; factorisation and
 * solve are decoupled so that many right-hand sides reuse one factorisation (Section 4.2.3).
 *
 * Conventions for every call below:
 *   - All vectors are in the caller's point order, column-major (N x nrhs, leading dimension
 *     ld >= N), FP64. Pointers named *_dev are CUDA device pointers, *_host are host pointers.
 *   - The handle owns all device memory it allocates; the caller owns every pointer it passes.
 *   - No exception crosses the ABI. A failing call returns a status; ifmm_last_error() gives a
 *     one-line message. A failed factorisation leaves the handle valid but unfactored.
 *   - All device work is queued on the stream given to ifmm_build (NULL = legacy default
 *     stream); calls that return results to the host synchronise that stream.
 *   - A handle belongs to the device that was current at ifmm_build. Every call on it makes that
 *     device current for its duration and gives the caller's current device back on return.
 *   - Not thread-safe per handle: calls on one handle must not overlap.
 */
#ifndef IFMM_H
#define IFMM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ifmm_handle* ifmm_h;

typedef enum {
    IFMM_OK = 0,
    IFMM_ERR_INVALID_ARG = 1,    /* bad size, pointer, parameter or point outside the root box */
    IFMM_ERR_CUDA = 2,           /* a CUDA runtime call failed (message in ifmm_last_error)   */
    IFMM_ERR_OOM = 3,            /* device allocation failed                                   */
    IFMM_ERR_SINGULAR_PIVOT = 4, /* a pivot block P2P/P2M (Eqs. P2P(i,k), P2M(i,k)) is singular */
    IFMM_ERR_RANK_OVERFLOW = 5,  /* a box basis needed more than r_cap directions             */
    IFMM_ERR_NOCONV = 6,         /* iterative refinement did not reach refine_tol             */
    IFMM_ERR_TIMEOUT = 7,        /* a bounded device wait (on the tensor cores) ran out       */
    IFMM_ERR_STATE = 8           /* call out of order (e.g. solve before factor)              */
} ifmm_status;

typedef enum {
    IFMM_K_INV_R = 0,            /* K(x, y) = 1 / |x - y|                                      */
    IFMM_K_EXP = 1,              /* K(x, y) = exp(-|x - y| / kparam[0])                        */
    IFMM_K_DEXP_DELL = 2,        /* K(x, y) = d/dl exp(-r / l) = (r / l^2) exp(-r / l), l = kparam[0],
                                    r = |x - y|: with diag = 0 its FMM matvec is dA~/dl of the
                                    IFMM_K_EXP matrix (the Chebyshev nodes and bases do not depend
                                    on l), the parameter derivative an adjoint gradient needs    */
    /* the regularised kernels of the numerical benchmarks (Section 5), a = kparam[0] (0.001 there),
       used with diag = 1 (Eq. "main_Solving_Equation"); each is 0 at r = 0                      */
    IFMM_K_LOG_REG = 3,          /* r (log r - 1) / (a (log a - 1)) for r < a, ln r / ln a beyond  */
    IFMM_K_INV_REG = 4,          /* r / a for r < a, a / r beyond                                  */
    IFMM_K_R2LOG_REG = 5         /* r^3 (3 log r - 1) / (a^3 (3 log a - 1)) for r < a,
                                    r^2 ln r / (a^2 ln a) beyond                                   */
} ifmm_kernel;

typedef enum {
    IFMM_FP64 = 0,               /* every step in FP64                                         */
    IFMM_MIXED = 1,              /* FP32 Schur updates, panels and compression; FP64 pivot
                                    blocks, residual matvec and refinement update              */
    IFMM_MIXED_SOLVE = 2         /* FP64 elimination; the solve phase on the FP32 pipe in
                                    double-float arithmetic (pairs of FP32, ~48-bit significand):
                                    the replay of double-float copies of the factors and the FMM
                                    matvec inside GMRES; the residual that may end the solve
                                    is an FP64 matvec (restarts that only seed the next cycle
                                    take the double-float one), updates are FP64              */
} ifmm_precision;

typedef struct {
    int dim;              /* space dimension: 2 (quadtree) or 3 (octree: Section 4.2 extends the
                             method to any dimension; 27 neighbours and up to 189 interaction-list
                             boxes per box, 27 colours). 3 requires cheb_p <= 4, an explicit
                             depth <= 6 and tc_products = 0                                        */
    int depth;            /* leaf level kappa of the uniform tree, 2 <= depth <= 10; 0 = automatic
                             (see leaf_max; 2D only)                                              */
    int cheb_p;           /* Chebyshev nodes per dimension (Section 5), 1..8; initial box rank p^dim */
    int r_cap;            /* largest rank any box basis may reach (if > 0, at least cheb_p^2);
                             <= 0: only the box size n_i                                          */
    double eps;           /* compression tolerance of the fill-in (Section 5), >= 0              */
    double diag;          /* diagonal A_ii, finite (the paper's Eq. "main_Solving_Equation" uses 1) */
    double kparam[4];     /* kernel parameters: kparam[0] > 0 for every kernel but IFMM_K_INV_R
                             (the length scale l of IFMM_K_EXP / IFMM_K_DEXP_DELL, the a of the
                             benchmark kernels)                                                   */
    double box[3];        /* root box x0, y0, side; side <= 0 selects the unit square (cube) with
                             its corner at the origin. 3D: the cube [x0, x0 + side] x [y0, y0 + side]
                             x [z0, z0 + side]                                                    */
    int precision;        /* ifmm_precision                                                       */
    int tau_ref;          /* compression threshold reference: 0 = the fill's own largest column
                             norm; 1 = the matrix scale s_A (largest column norm of the leaf
                             diagonal blocks), i.e. an absolute tolerance eps * s_A at every level;
                             2 = the scale of the level (largest column norm of its diagonal blocks
                             at the start of the level)                                           */
    double refine_tol;    /* FP64 refinement stops when the preconditioned residual
                             max_j ||M^{-1}(b_j - A~ x_j)|| / ||x_j|| (an estimate of the relative error,
                             M^{-1} = the IFMM solve) is <= refine_tol; 0 disables refinement         */
    int refine_maxit;     /* limit on preconditioned matvecs (IFMM_ERR_NOCONV past it)            */
    int refine_restart;   /* 1..200: GMRES(refine_restart) left-preconditioned by the IFMM solve;
                             0: classical refinement x += M^{-1}(b - A~ x)                          */
    double refine_inner;  /* IFMM_MIXED_SOLVE: a GMRES cycle (double-float products) ends once its error
                             estimate has fallen by this factor, and the next cycle starts from a
                             recomputed residual (double-float; FP64 once the estimate has reached
                             refine_tol, and only an FP64 one ends the solve); <= 0 selects 1e-4    */
    int leaf_max;         /* depth = 0: the build takes the smallest depth whose fullest leaf holds
                             at most leaf_max points (ifmm_auto_depth)                           */
    int tc_products;      /* IFMM_MIXED_SOLVE, products in FP64 accuracy on the tensor cores (the
                             digit-split product of ifmm_tc_dgemm): 1 = the replay of the solve
                             (FP64 vectors; the factors split into digits once, after the
                             factorisation); 2 = the replay and the Schur-update products of the
                             elimination; 0 (default) = neither: double-float replay and products
                             on the FP32 pipe. Range 0..2                                        */
    double svd_eps;       /* Chebyshev interpolation followed by SVD compression (Section 5): > 0
                             projects every level's p^2 Chebyshev coefficients onto the leading
                             left singular vectors of the level's M2L kernel matrices over the 40
                             interaction offsets (with the parent level's kept directions, so the
                             bases stay nested), keeping sigma_j > svd_eps * sigma_1; the kept
                             counts are ifmm_stats.svd_ranks. Meant for kernels of x - y alone
                             (all of ifmm_kernel). 0 (default): no truncation. Range [0, 1)   */
    double z0;            /* dim 3: lower z of the root cube (0 by default)                      */
} ifmm_params;

typedef struct {
    int64_t n_points;
    int depth;
    int max_rank;          /* r_m of the paper's tables: largest box rank after factorisation   */
    int rank_overflows;    /* 1 if some box basis was cut at r_cap                              */
    int refine_iters;      /* solves performed by the last ifmm_solve                            */
    double t_build_ms, t_factor_ms, t_solve_ms;   /* t_a, t_f, t_s of Table "table_notations"    */
    double factor_flops;   /* algorithmic flops of the last factorisation at the actual ranks    */
    double schur_flops;    /* algorithmic flops of the Schur-update launches                       */
    double schur_bytes;    /* algorithmic bytes of the Schur-update launches (blocks read + written) */
    double kernel_ms[5];   /* device time (CUDA events on the handle's stream) of the pivot, panel,
                              Schur, compression and redirect launches of the last factorisation     */
    int kernel_launches[5];/* launches of each of those five kernels in the last factorisation      */
    double kernel_flops[5];/* algorithmic flops of each of those five kernels (actual sizes)         */
    double level_ms[16];   /* device time of the five kernels per tree level (index = level)       */
    double last_update;    /* max_j ||dx_j|| / ||x_j|| of the last refinement step                 */
    double last_residual;  /* max_j ||b_j - A~ x_j|| / ||b_j|| before the last refinement step     */
    int64_t device_bytes;  /* device memory held by the handle                                     */
    int64_t launches_factor; /* kernels launched by the last ifmm_factor                           */
    int64_t launches_solve;  /* kernels launched by the last ifmm_solve / ifmm_solve_host          */
    double compress_proj_flops; /* the part of kernel_flops[3] spent projecting the fill onto the
                              complement of the old basis (products; double-float in
                              IFMM_MIXED_SOLVE); the rest is the pivoted Gram-Schmidt              */
    int svd_ranks[16];     /* singular vectors kept per level (index = level) with svd_eps > 0;
                              0 otherwise                                                           */
    double compress_reorth_flops; /* the part of kernel_flops[3] spent re-orthogonalising each new
                              direction against the basis (FP64 in every mode); the rest beyond
                              compress_proj_flops is the Gram-Schmidt's column work (dot products,
                              updates and norms: double-float in IFMM_MIXED_SOLVE, else FP64)        */
} ifmm_stats;

/* Default parameters: dim 2, depth 3, cheb_p 4, r_cap 0, eps 1e-10, diag 1, unit square,
 * FP64, tau_ref 1, no refinement (refine_maxit 100, refine_restart 60, refine_inner 1e-4),
 * leaf_max 64, tc_products 0, svd_eps 0, z0 0. */
void ifmm_default_params(ifmm_params* p);

/* Smallest depth 2..10 of the uniform quadtree (Section 4.2: boxes of level k form a 2^k x 2^k
 * grid of the root box) whose fullest leaf holds at most leaf_max points; 10 if none. pts_host:
 * N x 2 row-major host array; box: {x0, y0, side} or NULL for the unit square (side <= 0 also
 * selects it). Host only (no device call). Returns -1 for invalid arguments. */
int ifmm_auto_depth(const double* pts_host, int64_t N, const double* box, int leaf_max);

/* Build the tree, the Chebyshev operators and their orthonormal nested bases (assembly time t_a).
 * pts_host: N x dim row-major FP64 host array (x0, y0[, z0], x1, y1[, z1], ...), copied; N >= 1.
 * kernel:   ifmm_kernel. p: parameters (copied). stream: cudaStream_t or NULL.
 * out:      receives the handle (NULL on failure).
 * Tree and lists: Section 4.2, Table "table_cluster"; operators: Table "table_FMM_operators";
 * Chebyshev interpolation: Section 5. Errors: INVALID_ARG (N outside 1..2^31-1, a non-finite
 * coordinate or a point outside the root box, a parameter outside the ranges above), CUDA, OOM. */
ifmm_status ifmm_build(const double* pts_host, int64_t N, int kernel, const ifmm_params* p,
                       void* stream, ifmm_h* out);

/* Eliminate every box, levels kappa..2 (Algorithm 1), then factor the level-1 system
 * (factorisation time t_f). Calling it again discards the previous factorisation and recomputes
 * it from the operators of the build. Errors: SINGULAR_PIVOT, CUDA, OOM (handle left
 * unfactored); RANK_OVERFLOW (the factorisation completed and is usable, but some box basis was
 * cut at r_cap, so the solve is coarser than eps). */
ifmm_status ifmm_factor(ifmm_h h);

/* x = A~^{-1} b by forward replay of the eliminations, the level-1 solve and back substitution
 * (Algorithm 2); when refine_tol > 0 that solve is the preconditioner M^{-1} of an iterative
 * refinement (GMRES or classical) on A~ x = b whose residuals use the FMM matvec (solve time t_s).
 * b_dev, x_dev: device FP64, column-major, leading dimension ld >= N; 1 <= nrhs <= 1024; b and x
 * must not overlap; rows N..ld-1 of x are not written. Errors: STATE (not factored), INVALID_ARG,
 * NOCONV (x still holds the last iterate), CUDA, OOM. */
ifmm_status ifmm_solve(ifmm_h h, const double* b_dev, double* x_dev, int nrhs, int64_t ld);

/* x = A~^{-T} b: the transposed system, as needed by an adjoint (a gradient through the solve).
 * Every kernel of this library is symmetric and the build keeps A~ = A~^T (P2P_ji = P2P_ij^T,
 * M2L_ji = M2L_ij^T, L2P = P2M^T, Table "table_FMM_operators"), and the elimination compresses the
 * fill of a box with one basis for its row and its column, so the factors invert a symmetric
 * matrix and the transposed solve replays them exactly as ifmm_solve does (Algorithm 2).
 * Arguments, layout, refinement and errors are those of ifmm_solve. */
ifmm_status ifmm_solve_T(ifmm_h h, const double* b_dev, double* x_dev, int nrhs, int64_t ld);

/* Batched factorisation of n independent systems (no counterpart in the paper, which solves one
 * system; the batched workload of many uneven systems). A native scheduler gives the systems,
 * largest N first, to `workers` host threads (<= 0: min(n, 16)), each to the thread with the least
 * work so far; a thread factors its systems one after another on their own handles' streams, so
 * handles built on distinct streams run concurrently on the GPU. status_out (n entries, may be
 * NULL) receives each ifmm_factor status; the call returns the first non-OK one (IFMM_OK when all
 * succeeded). Handles must be distinct; no other call may use them meanwhile. */
ifmm_status ifmm_factor_batch(ifmm_h* hs, int n, int workers, ifmm_status* status_out);

/* Batched ifmm_solve of n factored systems: system i solves nrhs[i] right-hand sides b_dev[i] into
 * x_dev[i] (device, column-major, leading dimension ld[i]); scheduling (by N x nrhs), streams,
 * statuses and return value as in ifmm_factor_batch. */
ifmm_status ifmm_solve_batch(ifmm_h* hs, int n, const double* const* b_dev, double* const* x_dev, const int* nrhs,
                             const int64_t* ld, int workers, ifmm_status* status_out);

/* Autotuner of the batched launches (no counterpart in the paper, which solves one system). The
 * panel and Schur-update launches of a colour split each box's (panel) or each neighbour pair's
 * (Schur) product over `split` thread blocks, each taking every split-th output tile. A
 * process-wide table maps a bucket -- (kernel, double-float products or not, ceil(log2) of the
 * level's largest block n, ceil(log2) of the launch's box count) -- to a split; a launch whose
 * bucket has no entry uses the fixed rule. A split changes only which block computes which tile,
 * so results are identical bit for bit whatever the table holds.
 * ifmm_autotune factors the given systems with ifmm_factor_batch (one warm-up, then once per
 * candidate split 1, 2, 4, 8, 16 for the panel and then the Schur launches), times every launch
 * with CUDA events, enters the fastest split of each bucket in the table and factors the systems
 * once more with it (they are left factored). Arguments and errors as ifmm_factor_batch; a
 * failing factorisation ends the tuning with the table unchanged.
 * ifmm_autotune_save / ifmm_autotune_load write / read the table as text (one bucket per line:
 * kernel df log2_nmax log2_boxes split; '#' lines are comments); load replaces the table and
 * rejects a malformed file (IFMM_ERR_INVALID_ARG, table unchanged). ifmm_autotune_clear empties
 * it; ifmm_autotune_size returns its number of entries. The table functions are host-only. */
ifmm_status ifmm_autotune(ifmm_h* hs, int n, int workers);
ifmm_status ifmm_autotune_save(const char* path);
ifmm_status ifmm_autotune_load(const char* path);
void ifmm_autotune_clear(void);
int ifmm_autotune_size(void);

/* Largest thread-block cluster over which one fill compression of Algorithm 1 (Section 4.2) may
 * be spread (1, 2, 4, 8 or 16; default 16, where the device can schedule it, else 8;
 * process-wide, read at each factorisation launch). Where a
 * colour has few boxes (the upper levels of the tree) the blocks of a cluster each take a slice
 * of the stacked fill's columns; the arithmetic per column is the same as with one block, so
 * ranks, bases and solutions are the same bit for bit for every setting. 1 turns the clusters
 * off. Errors: INVALID_ARG for any other value (setting unchanged). Host-only. */
ifmm_status ifmm_set_compress_cluster(int max_blocks);

/* As ifmm_solve with host buffers: copies b in and x out inside the call (one copy per column, or
 * one for the block when ld = N). Page-locked host buffers (cudaHostAlloc or pinned tensors) copy
 * at the link's rate; pageable ones are staged by the driver, several times slower. */
ifmm_status ifmm_solve_host(ifmm_h h, const double* b_host, double* x_host, int nrhs, int64_t ld);

/* y = A~ x with the FP64 FMM operators of the build: P2M, M2M, M2L, L2L, L2P and P2P
 * (Table "table_FMM_operators"). x_dev, y_dev: device FP64, column-major, leading dimension
 * ld >= N. Errors: INVALID_ARG, CUDA. */
ifmm_status ifmm_matvec(ifmm_h h, const double* x_dev, double* y_dev, int nrhs, int64_t ld);

/* y = A~ x exactly as ifmm_matvec, but without allocating any device memory. This call has no
 * counterpart in the paper; it serves callers that must not allocate: an application whose
 * device memory is owned by another allocator (a framework's caching pool, a fixed budget), or a
 * latency-sensitive loop in which an allocation would stall the device. ifmm_matvec allocates
 * its intermediate vectors in the handle on first use; this variant keeps them in one fixed
 * 32 MiB array compiled into the library (every GPU that loads the library holds those 32 MiB
 * until the process exits). Limit: 16 N nrhs + 16 nrhs p^2 (4^2 + ... + 4^depth) bytes, each
 * piece rounded up to 256 bytes, must fit in 32 MiB; larger calls return IFMM_ERR_INVALID_ARG
 * with the size in ifmm_last_error. The first call for a device (the handle's device, made current
 * by the call) looks up the array's device address on that device; make that first call before
 * any stream capture. All calls
 * share the array and each call overwrites it: calls that overlap on the GPU (two streams, two
 * threads, two handles on one device) race and must be serialised by the caller. Arguments,
 * layout and the other errors are those of ifmm_matvec; the call synchronises the handle's
 * stream. */
ifmm_status ifmm_matvec_noalloc(ifmm_h h, const double* x_dev, double* y_dev, int nrhs, int64_t ld);

/* C = A B in FP64 accuracy on the tensor cores: the product kernel of the Schur-complement update
 * A[rho, gamma] -= C_rho X_gamma of Algorithm 1 on its own. Each row of A and column of B is scaled
 * by a power of two and cut into eight 7-bit digits; the 36 digit products of weight <= 7 run as
 * bf16 tcgen05 MMAs whose FP32 accumulators hold exact integers, combined in 64-bit integer
 * arithmetic (relative error about 2^-52 of |A| |B|; exact when every entry has at most 53
 * significant bits within 56 bits of its row's or column's largest entry and the exact products and
 * sums fit in FP64). A (M x K, leading dimension lda >= K), B (K x N, ldb >= N), C (M x N, ldc >= N): device
 * pointers, row-major, FP64; C must not overlap A or B. stream: cudaStream_t or NULL; the call
 * synchronises it. Entries below 2^-1022 are flushed to zero. Errors: INVALID_ARG, CUDA, TIMEOUT
 * (a bounded wait on the tensor cores ran out; C is then undefined). */
ifmm_status ifmm_tc_dgemm(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                          int M, int N, int K, void* stream);

/* Final ranks of the boxes of one level 2..depth, grid order (ix + s (iy + s iz), s = 2^level), into
 * the host array out_host (2^(dim level) ints). Errors: STATE (not factored), INVALID_ARG. */
ifmm_status ifmm_get_ranks(ifmm_h h, int level, int* out_host);

/* Counters and timings of the handle into *s. Errors: INVALID_ARG (NULL argument). */
ifmm_status ifmm_get_stats(ifmm_h h, ifmm_stats* s);

/* One-line description of the last failure on this handle ("" if none). The string is owned
 * by the handle and valid until the next call on it. */
const char* ifmm_last_error(ifmm_h h);

/* Release the handle and all device memory it holds. NULL is ignored. */
void ifmm_destroy(ifmm_h h);

#ifdef __cplusplus
}
#endif
#endif
