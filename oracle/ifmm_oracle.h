/*
 * ifmm_oracle.h -- C interface of the CPU oracle for the Inverse Fast Multipole Method
 * (Ambikasaran & Darve, "The Inverse Fast Multipole Method", arXiv:1407.1572).
 *
 * TEST INFRASTRUCTURE ONLY. The oracle is a plain, slow FP64 restatement of the paper's
 * method (Section 4.2, Algorithms 1 and 2). It is called by the tests, by the package's
 * smoke check and by the bench's CPU-baseline leg, and by nothing in the product library.
 * It shares no code with the CUDA path.
 *
 * All vectors are in the caller's point order, column-major N x nrhs. Points are N x dim, row-major.
 * Return codes: 0 = ok, 1 = invalid argument, 4 = singular pivot, 8 = wrong call order.
 */
#ifndef IFMM_ORACLE_H
#define IFMM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_K_INV_R = 0, ORACLE_K_EXP = 1, ORACLE_K_DEXP_DELL = 2, ORACLE_K_POLY = 3,
       ORACLE_K_LOG_REG = 4, ORACLE_K_INV_REG = 5, ORACLE_K_R2LOG_REG = 6,
       ORACLE_K_R2 = 7 /* |x - y|^2: translation invariant, of exact separable rank 4 in 2D (a pin
                          of the SVD truncation) */ };

typedef struct {
    int depth;          /* leaf level kappa >= 2 of the uniform tree (<= 7 in 3D)              */
    int cheb_p;         /* Chebyshev nodes per dimension; initial rank p^dim (p <= 6 in 3D)     */
    int kernel;         /* ORACLE_K_*                                                           */
    int r_cap;          /* upper bound on any box rank (<= 0: no cap besides n_i)              */
    double eps;         /* relative compression tolerance of the fill-ins                      */
    double diag;        /* matrix diagonal A_ii                                                 */
    double kparam[4];   /* kernel parameters (EXP: kparam[0] = length scale)                   */
    double box[3];      /* root box: x0, y0, side length                                       */
    int order;          /* 0 = colour-major elimination order, 1 = Morton order                */
    int threads;        /* OpenMP threads for same-colour boxes (<= 0: default)                */
    int tau_ref;        /* compression threshold reference: 0 = eps * largest column norm of the
                           fill being compressed; 1 = eps * s_A, the largest column norm over the
                           leaf diagonal blocks (matrix scale); 2 = eps * the largest column norm
                           over the diagonal blocks P2P_ii^(k) of the level being eliminated      */
    double svd_eps;     /* > 0: Chebyshev interpolation followed by SVD compression (Section 5):
                           at every level k the p^2 Chebyshev coefficients are projected onto the
                           leading left singular vectors U_k of the level's M2L kernel matrices
                           [K(nodes_0, nodes_0 + h_k d)] over the 40 interaction offsets d, keeping
                           those with sigma_j > svd_eps * sigma_1 (translation-invariant kernels);
                           0: no truncation                                                       */
    int dim;            /* space dimension: 2 (quadtree; 0 means 2) or 3 (octree, Section 4.2's
                           extension to 3D: 27 neighbours, up to 189 interaction-list boxes, 27
                           colours, p^3 Chebyshev nodes); points are N x dim, row-major          */
    double z0;          /* dim 3: lower z of the root cube [box[0], +box[2]] x [box[1], +box[2]] x
                           [z0, z0 + box[2]]                                                      */
} oracle_params;

void* oracle_build(const double* pts, int64_t N, const oracle_params* prm);
void  oracle_destroy(void* h);
int   oracle_factor(void* h);
int   oracle_solve(void* h, const double* b, double* x, int nrhs);
int   oracle_matvec(void* h, const double* x, double* y, int nrhs);

/* dense N x N matrices, row-major, caller's point order (small N only) */
int   oracle_dense_tilde(void* h, double* A);         /* the FMM matrix via the nested operators    */
int   oracle_dense_tilde_direct(void* h, double* A);  /* same matrix, Chebyshev formula per level  */
int   oracle_dense_exact(void* h, double* A);         /* the kernel matrix A itself                */
int   oracle_extended_solve(void* h, const double* b, double* x, int nrhs); /* dense extended system */
int   oracle_dense_lu_solve(const double* A, int64_t n, const double* b, double* x, int nrhs);

/* introspection for the tests */
int   oracle_num_boxes(void* h, int level);
int   oracle_ranks(void* h, int level, int* out);          /* final ranks, grid order ix + s (iy + s iz) */
int   oracle_initial_ranks(void* h, int level, int* out);  /* ranks after orthonormalisation         */
int   oracle_leaf_counts(void* h, int* out);
int   oracle_perm(void* h, int64_t* out);                  /* tree position -> caller index           */
int   oracle_lists(void* h, int level, int box, int* nbr, int* n_nbr, int* inter, int* n_inter);
int   oracle_order(void* h, int level, int* out);          /* elimination order (grid indices)       */
/* stats: [0] flops, [1] bytes, [2] compressions (augmenting events), [3] rank overflows,
 *        [4] max rank, [5] eliminations, [6] directions added, [7] factor seconds,
 *        [8] matrix scale s_A (largest column norm over the leaf diagonal blocks)             */
int   oracle_stats(void* h, double* out, int nout);

/* primitives used as pins */
void  oracle_cheb_nodes(int p, double* t);
void  oracle_lagrange(int p, double t, double* out);
int   oracle_kernel_eval(const oracle_params* prm, const double* a, const double* b, double* out);
/* out[i * n + j] = K(P_i, Q_j) for m points P and n points Q (row-major, dim coordinates each),
 * no diagonal; a and b of oracle_kernel_eval likewise hold dim coordinates */
int   oracle_kernel_matrix(const oracle_params* prm, const double* P, int64_t m, const double* Q, int64_t n,
                           double* out);

/* The SVD of level k's M2L kernel matrices (the svd_eps truncation above), computed whatever the
 * handle's svd_eps: sigma (p^2, descending) and U (p^2 x p^2, row-major, column j = the left
 * singular vector of sigma_j, its entry of largest magnitude positive). Returns the number of
 * singular values above svd_eps * sigma_1 for the handle's svd_eps (p^2 when it is 0), -1 on bad
 * arguments. */
int   oracle_svd_basis(void* h, int level, double* U, double* sigma);

/* The compression step of reading R2 alone: append to W (n x r, row-major, orthonormal columns;
 * NULL when r = 0) the directions of S (n x m, row-major) that W misses, by pivoted Gram-Schmidt
 * on (I - W W^T) S with threshold eps * ref (ref > 0) or eps * (largest column norm of S)
 * (ref <= 0), at most cap columns in all (cap <= 0: n). Wout receives the extended basis
 * (n x (r + added), row-major; room for n x n). Returns the number of appended directions (-1 on
 * bad arguments); *overflow = 1 if the cap cut it. */
int   oracle_augment_basis(const double* W, int n, int r, const double* S, int m, double eps, double ref, int cap,
                           double* Wout, int* overflow);

#ifdef __cplusplus
}
#endif
#endif
