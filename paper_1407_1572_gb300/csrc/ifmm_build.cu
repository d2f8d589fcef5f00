// ifmm_build.cu -- tree, Chebyshev operators and the FP64 FMM matvec, sm_103a.
//
// Build (assembly time t_a of Table "table_notations"):
//   points -> leaf keys (Morton code of the leaf, Section 4.2: uniform 2^d tree, d = 2 or 3,
//   Morton order) -> bitonic sort -> tree order, leaf counts;
//   leaf bases V_b[a, m] = S_m(x_a), the tensor Lagrange basis at p^d first-kind Chebyshev
//   nodes of the leaf (Section 5), orthonormalised by column-pivoted Householder QR, V = Q Rt;
//   parent bases: the stacked children transfers Rt_c T_c (T_c[m', m] = parent basis m at child
//   node m'), orthonormalised the same way;
//   M2L_bq = Rt_b K(nodes_b, nodes_q) Rt_q^T for q in the interaction list I_b;
//   leaf P2P_bq = K(x_a, x_c) for q in N_b, with the diagonal A_aa on the same point.
// Matvec y = A~ x (Table "table_FMM_operators"): P2M, M2M, M2L, L2L, L2P and P2P in FP64.
#include <atomic>
#include <cstdio>

#include "ifmm_common.cuh"
#include "ifmm_internal.h"

namespace ifmm {

// Morton code of a cell: the bits of x, y (and z) interleaved, d bits per level
IFMM_DEVINL unsigned long long morton_code(Cell c, int dim) {
    unsigned long long m = 0;
    for (int bit = 0; bit < 10; ++bit) {
        m |= (unsigned long long)((c.x >> bit) & 1) << (dim * bit);
        m |= (unsigned long long)((c.y >> bit) & 1) << (dim * bit + 1);
        if (dim == 3) m |= (unsigned long long)((c.z >> bit) & 1) << (dim * bit + 2);
    }
    return m;
}
IFMM_DEVINL Cell morton_cell(unsigned long long m, int dim) {
    Cell c{0, 0, 0};
    for (int bit = 0; bit < 10; ++bit) {
        c.x |= (int)((m >> (dim * bit)) & 1) << bit;
        c.y |= (int)((m >> (dim * bit + 1)) & 1) << bit;
        if (dim == 3) c.z |= (int)((m >> (dim * bit + 2)) & 1) << bit;
    }
    return c;
}

IFMM_DEVINL double kernel_eval(int kernel, double kparam0, double ax, double ay, double az, double bx, double by,
                               double bz) {
    const double dx = ax - bx, dy = ay - by, dz = az - bz;
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (kernel == 0) return 1.0 / r;
    if (kernel == 2) return r / (kparam0 * kparam0) * exp(-r / kparam0);  // d/dl of exp(-r / l)
    if (kernel >= 3) {
        // the regularised benchmark kernels of Section 5 (a = kparam0), each 0 at r = 0
        const double a = kparam0;
        if (kernel == 4) return r < a ? r / a : a / r;
        if (r == 0.0) return 0.0;
        if (kernel == 3) return r < a ? r * (log(r) - 1.0) / (a * (log(a) - 1.0)) : log(r) / log(a);
        return r < a ? r * r * r * (3.0 * log(r) - 1.0) / (a * a * a * (3.0 * log(a) - 1.0))
                     : r * r * log(r) / (a * a * log(a));
    }
    return exp(-r / kparam0);
}

// ---------------------------------------------------------------------------------------------
// tree
// ---------------------------------------------------------------------------------------------
__global__ void k_leaf_keys(const double* pts, int64_t N, int depth, int dim, double x0, double y0, double z0,
                            double L, unsigned long long* keys, int64_t npad, int* status) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npad) return;
    if (t >= N) { keys[t] = ~0ull; return; }
    const int side = 1 << depth;
    const double org[3] = {x0, y0, z0};
    int c[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) {
        double u = (pts[dim * t + i] - org[i]) / L;
        if (!(u >= 0.0 && u <= 1.0)) {
            atomicOr(status, DEV_ERR_RANGE);
            u = fmin(fmax(u, 0.0), 1.0);
        }
        c[i] = min((int)floor(u * side), side - 1);
    }
    const unsigned long long m = morton_code(Cell{c[0], c[1], c[2]}, dim);
    keys[t] = (m << 32) | (unsigned long long)t;
}

void launch_leaf_keys(const double* pts, int64_t N, int depth, int dim, double x0, double y0, double z0, double L,
                      unsigned long long* keys, int64_t npad, int* status, cudaStream_t st) {
    k_leaf_keys<<<(unsigned)((npad + 255) / 256), 256, 0, st>>>(pts, N, depth, dim, x0, y0, z0, L, keys, npad, status);
    count_launches(1);
}

__global__ void k_bitonic_step(unsigned long long* keys, int64_t npad, int64_t j, int64_t k) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    int64_t l = i ^ j;
    if (l <= i) return;
    unsigned long long a = keys[i], b = keys[l];
    bool up = (i & k) == 0;
    if ((a > b) == up) { keys[i] = b; keys[l] = a; }
}

// in-block stages (j < 1024) of the bitonic network in shared memory
__global__ void k_bitonic_local(unsigned long long* keys, int64_t npad, int64_t k, int64_t jstart) {
    __shared__ unsigned long long s[2048];
    const int64_t base = (int64_t)blockIdx.x * 2048;
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) s[t] = keys[base + t];
    __syncthreads();
    for (int64_t j = jstart; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
            int64_t i = base + t, l = i ^ j;
            if (l > i) {
                int tl = (int)(l - base);
                unsigned long long a = s[t], b = s[tl];
                bool up = (i & k) == 0;
                if ((a > b) == up) { s[t] = b; s[tl] = a; }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) keys[base + t] = s[t];
}

void launch_bitonic_sort(unsigned long long* keys, int64_t npad, cudaStream_t st) {
    for (int64_t k = 2; k <= npad; k <<= 1) {
        int64_t j = k >> 1;
        for (; j >= 1024 && j >= 1; j >>= 1)
            { k_bitonic_step<<<(unsigned)((npad + 255) / 256), 256, 0, st>>>(keys, npad, j, k); count_launches(1); }
        if (j >= 1) {
            if (npad >= 2048)
                { k_bitonic_local<<<(unsigned)(npad / 2048), 1024, 0, st>>>(keys, npad, k, j); count_launches(1); }
            else
                for (; j >= 1; j >>= 1)
                    { k_bitonic_step<<<(unsigned)((npad + 255) / 256), 256, 0, st>>>(keys, npad, j, k); count_launches(1); }
        }
    }
}

__global__ void k_scatter_sorted(const unsigned long long* keys, const double* pts, int64_t N, int dim, int64_t* perm,
                                 double* px, double* py, double* pz, int* leaf_count, int depth) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    unsigned long long key = keys[t];
    int64_t idx = (int64_t)(key & 0xffffffffull);
    const Cell c = morton_cell(key >> 32, dim);
    perm[t] = idx;
    px[t] = pts[dim * idx];
    py[t] = pts[dim * idx + 1];
    pz[t] = dim == 3 ? pts[dim * idx + 2] : 0.0;
    atomicAdd(&leaf_count[cell_index(c, 1 << depth)], 1);
}

void launch_scatter_sorted(const unsigned long long* keys, const double* pts, int64_t N, int dim, int64_t* perm,
                           double* px, double* py, double* pz, int* leaf_count, int depth, cudaStream_t st) {
    k_scatter_sorted<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(keys, pts, N, dim, perm, px, py, pz, leaf_count,
                                                                  depth);
    count_launches(1);
}

// ---------------------------------------------------------------------------------------------
// bases
// ---------------------------------------------------------------------------------------------
IFMM_DEVINL double lagrange1(int p, const double* t, int m, double x) {
    double v = 1.0;
    for (int j = 0; j < p; ++j)
        if (j != m) v *= (x - t[j]) / (t[m] - t[j]);
    return v;
}

// per leaf: V (n x r0) -> Q (rows of W0 in tree order), Rt, rank. Scratch in global memory:
// Ascr (n x r0) and Vscr (reflectors) at the leaf's tree rows. With the SVD compression (U, the
// leaf level's kept singular vectors, p^2 x rk in a p^2 x p^2 array, rk = *rsvd) the
// orthonormalised matrix is V U and Rt is mapped back to node values: Rt <- Rt U^T.
__global__ void __launch_bounds__(kThreads) k_leaf_basis(BuildArgs a, const double* px, const double* py,
                                                         const double* pz, const int64_t* leaf_start,
                                                         const int* leaf_count,
                                                         const double* cheb, double* W0, double* Rt, int* rank0,
                                                         double* Ascr, double* Vscr, const double* U,
                                                         const int* rsvd) {
    __shared__ double red[32];
    __shared__ int ired[32];
    __shared__ double beta[64];
    __shared__ int cperm[64];
    const int b = blockIdx.x;
    const int side = 1 << a.depth;
    const Cell cb = cell_of(b, side, a.dim);
    const int n = leaf_count[b];
    const int64_t s0 = leaf_start[b];
    const int p = a.p, r0 = a.r0;
    const double h = a.L / side;
    const double lx = a.x0 + cb.x * h, ly = a.y0 + cb.y * h, lz = a.z0 + cb.z * h;
    double* A = Ascr + s0 * r0;
    double* Q = W0 + s0 * r0;
    const int rk = U ? *rsvd : r0;
    double* S = U ? Q : A;   // the interpolation matrix; with U it is projected into A below
    for (int t = threadIdx.x; t < n * r0; t += blockDim.x) {
        int i = t / r0, m = t - i * r0;
        int mx = m % p, my = (m / p) % p, mz = m / (p * p);
        double ux = 2.0 * (px[s0 + i] - lx) / h - 1.0, uy = 2.0 * (py[s0 + i] - ly) / h - 1.0;
        double v = lagrange1(p, cheb, mx, ux) * lagrange1(p, cheb, my, uy);
        if (a.dim == 3) v *= lagrange1(p, cheb, mz, 2.0 * (pz[s0 + i] - lz) / h - 1.0);
        S[(size_t)i * r0 + m] = v;
    }
    if (U) {
        __syncthreads();
        for (int t = threadIdx.x; t < n * r0; t += blockDim.x) {
            int i = t / r0, j = t - i * r0;
            double v = 0.0;
            if (j < rk)
                for (int m = 0; m < r0; ++m) v += S[(size_t)i * r0 + m] * U[(size_t)m * r0 + j];
            A[t] = v;
        }
        __syncthreads();
    }
    double* R = Rt + (int64_t)b * r0 * r0;
    for (int t = threadIdx.x; t < r0 * r0; t += blockDim.x) R[t] = 0.0;
    for (int t = threadIdx.x; t < n * r0; t += blockDim.x) Q[t] = 0.0;
    __syncthreads();
    int rank = 0;
    if (n > 0) rank = cta_cpqr(A, n, rk, r0, 1e-13, Q, r0, R, r0, Vscr + s0 * r0, beta, cperm, red, ired);
    if (U && rank > 0) {
        // Rt U^T (rank x r0) through A, which the factorisation no longer needs (rank <= n)
        for (int t = threadIdx.x; t < rank * r0; t += blockDim.x) {
            int i = t / r0, m = t - i * r0;
            double v = 0.0;
            for (int j = 0; j < rk; ++j) v += R[(size_t)i * r0 + j] * U[(size_t)m * r0 + j];
            A[t] = v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < rank * r0; t += blockDim.x) R[t] = A[t];
    }
    if (threadIdx.x == 0) rank0[b] = rank;
}

void launch_leaf_basis(const BuildArgs& a, const double* px, const double* py, const double* pz,
                       const int64_t* leaf_start, const int* leaf_count, const double* cheb, double* W0, double* Rt,
                       int* rank0, int max_n, const double* U, const int* rsvd, cudaStream_t st) {
    (void)max_n;
    // scratch lives in the second half of W0's allocation (the caller allocates 3 N r0 doubles)
    double* Ascr = W0 + a.N * a.r0;
    double* Vscr = W0 + 2 * a.N * a.r0;
    k_leaf_basis<<<1 << (a.dim * a.depth), kThreads, 0, st>>>(a, px, py, pz, leaf_start, leaf_count, cheb, W0, Rt,
                                                              rank0, Ascr, Vscr, U, rsvd);
    count_launches(1);
}

// per parent P at level k: Z stacks the rows (Rt_c T_c)[t, :], t < rank_c, of the 2^d children
// (Morton order) -> Z = Q Rt_P; Q is scattered into W0_P with rows c*r0 + t (zero rows for the
// components a child does not have). Scratch: Z, reflectors and the compact Q, each 2^d r0 x r0 per box,
// in the tail of the level's W0 allocation. With the SVD compression (U, rsvd of this level, as in
// k_leaf_basis) Z is orthonormalised in U's coordinates, Z U, and Rt mapped back, Rt U^T.
__global__ void __launch_bounds__(kThreads) k_parent_basis(BuildArgs a, int k, const double* Rt_child,
                                                           const int* rank_child, const double* Tc, double* W0,
                                                           double* Rt, int* rank0, double* Zscr, double* Vscr,
                                                           double* Qscr, const double* U, const int* rsvd) {
    __shared__ double red[32];
    __shared__ int ired[32];
    __shared__ double beta[64];
    __shared__ int cperm[64];
    const int b = blockIdx.x;
    const int side = 1 << k, cs = side << 1;
    const Cell cb = cell_of(b, side, a.dim);
    const int r0 = a.r0, nk = 1 << a.dim;
    int cg[8], off[9];
    off[0] = 0;
    for (int c = 0; c < nk; ++c) {
        cg[c] = cell_index(child_cell(cb, c), cs);
        off[c + 1] = off[c] + rank_child[cg[c]];
    }
    const int m = off[nk];
    const int rk = U ? *rsvd : r0;
    double* Z = Zscr + (int64_t)b * nk * r0 * r0;
    double* Q = Qscr + (int64_t)b * nk * r0 * r0;
    double* Z0 = U ? Q : Z;   // the stacked rows; with U projected into Z below
    for (int t = threadIdx.x; t < m * r0; t += blockDim.x) {
        int row = t / r0, col = t - row * r0;
        int c = 0;
        while (row >= off[c + 1]) ++c;
        int i = row - off[c];
        const double* Rc = Rt_child + (int64_t)cg[c] * r0 * r0;
        const double* T = Tc + (int64_t)c * r0 * r0;
        double v = 0.0;
        for (int l = 0; l < r0; ++l) v += Rc[(size_t)i * r0 + l] * T[(size_t)l * r0 + col];
        Z0[t] = v;
    }
    if (U) {
        __syncthreads();
        for (int t = threadIdx.x; t < m * r0; t += blockDim.x) {
            int row = t / r0, j = t - row * r0;
            double v = 0.0;
            if (j < rk)
                for (int l = 0; l < r0; ++l) v += Z0[(size_t)row * r0 + l] * U[(size_t)l * r0 + j];
            Z[t] = v;
        }
    }
    double* R = Rt + (int64_t)b * r0 * r0;
    for (int t = threadIdx.x; t < r0 * r0; t += blockDim.x) R[t] = 0.0;
    double* W = W0 + (int64_t)b * nk * r0 * r0;
    for (int t = threadIdx.x; t < nk * r0 * r0; t += blockDim.x) W[t] = 0.0;
    __syncthreads();
    int rank = 0;
    if (m > 0) rank = cta_cpqr(Z, m, rk, r0, 1e-13, Q, r0, R, r0, Vscr + (int64_t)b * nk * r0 * r0, beta, cperm, red, ired);
    if (U && rank > 0) {
        for (int t = threadIdx.x; t < rank * r0; t += blockDim.x) {   // Rt U^T through Z (rank <= m)
            int i = t / r0, l = t - i * r0;
            double v = 0.0;
            for (int j = 0; j < rk; ++j) v += R[(size_t)i * r0 + j] * U[(size_t)l * r0 + j];
            Z[t] = v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < rank * r0; t += blockDim.x) R[t] = Z[t];
    }
    for (int t = threadIdx.x; t < m * rank; t += blockDim.x) {
        int row = t / rank, j = t - row * rank;
        int c = 0;
        while (row >= off[c + 1]) ++c;
        W[(size_t)(c * r0 + row - off[c]) * r0 + j] = Q[(size_t)row * r0 + j];
    }
    if (threadIdx.x == 0) rank0[b] = rank;
}

void launch_parent_basis(const BuildArgs& a, int k, const double* Rt_child, const int* rank_child,
                         const double* Tc, double* W0, double* Rt, int* rank0, const double* U, const int* rsvd,
                         cudaStream_t st) {
    int64_t nb = 1ll << (a.dim * k);
    const int64_t nk = 1 << a.dim;
    double* Zscr = W0 + nb * nk * a.r0 * a.r0;
    double* Vscr = W0 + 2 * nb * nk * a.r0 * a.r0;
    double* Qscr = W0 + 3 * nb * nk * a.r0 * a.r0;
    k_parent_basis<<<(unsigned)nb, kThreads, 0, st>>>(a, k, Rt_child, rank_child, Tc, W0, Rt, rank0, Zscr, Vscr,
                                                      Qscr, U, rsvd); count_launches(1);
}

// The SVD compression of the Chebyshev interpolation (Section 5, "Chebyshev interpolation followed by
// SVD"), one level per launch, one CTA, top level first. G (m x r0, global scratch) stacks
// K_d^T for the interaction offsets d of a box (2 <= max_i |d_i| <= 3: 40 in 2D, 316 in 3D;
// K_d[i, l] = K(node_i, node_l + h d), h the box side
// of level k) and, below the top level, the parent's kept directions seen from each child position,
// (T_c U_{k-1} Sigma_{k-1})^T, so that the kept bases stay nested. G = Q R by Householder QR
// (cta_cpqr, no cut), then a one-sided Jacobi SVD of R in shared memory: in each round the r0
// columns form r0/2 disjoint pairs (a round-robin tournament), one warp per pair rotates its two
// columns (and those of V) orthogonal; sweeps repeat until no pair has |r_i . r_j| > 1e-15 |r_i| |r_j|
// (at most 60). sigma_j = |r_j|; U = V with columns sorted by sigma descending (ties by index),
// each column's entry of largest magnitude made positive; *rk = #{sigma_j > svd_eps sigma_1}, >= 1.
// U: r0 x r0 row-major; sig: r0. Up, sp, rp: the parent level's U, sigma and kept count (null at
// the top level). Shared memory: R and V, 2 r0^2 doubles.
__global__ void __launch_bounds__(kThreads) k_svd_level(BuildArgs a, int k, double svd_eps, const double* cheb,
                                                        const double* Tc, const double* Up, const double* sp,
                                                        const int* rp_dev, double* U, double* sig, int* rk,
                                                        double* G, double* Qs, double* Vs) {
    extern __shared__ double ssm[];
    __shared__ double red[32];
    __shared__ int ired[32];
    __shared__ double beta[64];
    __shared__ int cperm[64];
    __shared__ int offs[316];
    __shared__ double snorm[64];
    __shared__ int s_rot;
    const int r0 = a.r0, p = a.p;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double h = a.L / (double)(1 << k);
    const int rp = Up ? *rp_dev : 0;
    const int noff = a.dim == 3 ? 316 : 40, nk = 1 << a.dim;
    const int m = noff * r0 + nk * rp;
    if (threadIdx.x == 0) {
        int o = 0;
        for (int dz = (a.dim == 3 ? -3 : 0); dz <= (a.dim == 3 ? 3 : 0); ++dz)
            for (int dy = -3; dy <= 3; ++dy)
                for (int dx = -3; dx <= 3; ++dx)
                    if (max(abs(dx), max(abs(dy), abs(dz))) >= 2) offs[o++] = (dx + 3) + 7 * (dy + 3) + 49 * (dz + 3);
    }
    __syncthreads();
    auto node = [&](int m_, int c) { return 0.5 * (cheb[c == 0 ? m_ % p : (c == 1 ? (m_ / p) % p : m_ / (p * p))] + 1.0); };
    for (int t = threadIdx.x; t < noff * r0 * r0; t += blockDim.x) {
        const int o = t / (r0 * r0), l = (t / r0) % r0, i = t % r0;
        const int dx = offs[o] % 7 - 3, dy = (offs[o] / 7) % 7 - 3, dz = offs[o] / 49 - 3;
        const double az = a.dim == 3 ? node(i, 2) * h : 0.0, cz = a.dim == 3 ? (node(l, 2) + dz) * h : 0.0;
        G[t] = kernel_eval(a.kernel, a.kparam0, node(i, 0) * h, node(i, 1) * h, az, (node(l, 0) + dx) * h,
                           (node(l, 1) + dy) * h, cz);
    }
    for (int t = threadIdx.x; t < nk * rp * r0; t += blockDim.x) {
        const int c = t / (rp * r0), j = (t / r0) % rp, i = t % r0;
        const double* T = Tc + (size_t)c * r0 * r0;
        double v = 0.0;
        for (int l = 0; l < r0; ++l) v += T[(size_t)i * r0 + l] * Up[(size_t)l * r0 + j];
        G[(size_t)noff * r0 * r0 + t] = v * sp[j];
    }
    double* R = ssm;             // r0 x r0
    double* V = ssm + r0 * r0;   // r0 x r0
    for (int t = threadIdx.x; t < r0 * r0; t += blockDim.x) {
        R[t] = 0.0;
        V[t] = (t / r0 == t % r0) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int rank = cta_cpqr(G, m, r0, r0, 0.0, Qs, r0, R, r0, Vs, beta, cperm, red, ired);
    const int ne = r0 + (r0 & 1);   // players of the tournament; player r0 (odd r0) sits out
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        for (int round = 0; round < ne - 1; ++round) {
            for (int slot = warp; slot < ne / 2; slot += nw) {
                const int pa = slot, pb = ne - 1 - slot;   // positions; position 0 holds player 0
                const int i = pa == 0 ? 0 : (pa - 1 + round) % (ne - 1) + 1;
                const int j = (pb - 1 + round) % (ne - 1) + 1;
                if (i >= r0 || j >= r0) continue;
                double aa = 0.0, bb = 0.0, cc = 0.0;
                for (int q = lane; q < rank; q += 32) {
                    const double ri = R[q * r0 + i], rj = R[q * r0 + j];
                    aa += ri * ri; bb += rj * rj; cc += ri * rj;
                }
                aa = warp_sum(aa); bb = warp_sum(bb); cc = warp_sum(cc);
                if (cc == 0.0 || fabs(cc) <= 1e-15 * sqrt(aa * bb)) continue;
                const double zeta = (bb - aa) / (2.0 * cc);
                const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
                for (int q = lane; q < r0; q += 32) {
                    const double ri = R[q * r0 + i], rj = R[q * r0 + j];
                    R[q * r0 + i] = cs * ri - sn * rj;
                    R[q * r0 + j] = sn * ri + cs * rj;
                    const double vi = V[q * r0 + i], vj = V[q * r0 + j];
                    V[q * r0 + i] = cs * vi - sn * vj;
                    V[q * r0 + j] = sn * vi + cs * vj;
                }
                if (lane == 0) s_rot = 1;
            }
            __syncthreads();
        }
        const int rot = s_rot;
        __syncthreads();
        if (!rot) break;
    }
    for (int j = warp; j < r0; j += nw) {
        double ss = 0.0;
        for (int q = lane; q < r0; q += 32) ss += R[q * r0 + j] * R[q * r0 + j];
        ss = warp_sum(ss);
        if (lane == 0) snorm[j] = sqrt(ss);
    }
    __syncthreads();
    for (int j = warp; j < r0; j += nw) {
        int pos = 0;
        for (int i = 0; i < r0; ++i) pos += (snorm[i] > snorm[j] || (snorm[i] == snorm[j] && i < j)) ? 1 : 0;
        double best = -1.0;
        int bi = 0;
        for (int q = 0; q < r0; ++q)
            if (fabs(V[q * r0 + j]) > best) { best = fabs(V[q * r0 + j]); bi = q; }
        const double sg = V[bi * r0 + j] < 0.0 ? -1.0 : 1.0;
        for (int q = lane; q < r0; q += 32) U[(size_t)q * r0 + pos] = sg * V[q * r0 + j];
        if (lane == 0) sig[pos] = snorm[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double smax = 0.0;
        for (int j = 0; j < r0; ++j) smax = fmax(smax, snorm[j]);
        int cnt = 0;
        for (int j = 0; j < r0; ++j) cnt += snorm[j] > svd_eps * smax ? 1 : 0;
        *rk = cnt > 0 ? cnt : 1;
    }
}

void launch_svd_level(const BuildArgs& a, int k, double svd_eps, const double* cheb, const double* Tc,
                      const double* Up, const double* sp, const int* rp, double* U, double* sig, int* rk,
                      double* scratch, cudaStream_t st) {
    const size_t mmax = (size_t)(a.dim == 3 ? 324 : 44) * a.r0;
    double* G = scratch;
    double* Qs = G + mmax * a.r0;
    double* Vs = Qs + mmax * a.r0;
    const size_t smem = 2 * (size_t)a.r0 * a.r0 * sizeof(double);
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        cudaFuncSetAttribute(k_svd_level, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
        attr.store(true);
    }
    k_svd_level<<<1, kThreads, smem, st>>>(a, k, svd_eps, cheb, Tc, Up, sp, rp, U, sig, rk, G, Qs, Vs);
    count_launches(1);
}

size_t svd_scratch_doubles(int r0, int dim) { return (size_t)3 * (dim == 3 ? 324 : 44) * r0 * r0; }

// M2L_bq = Rt_b K(nodes_b, nodes_q) Rt_q^T for q in the interaction list of b
__global__ void __launch_bounds__(kThreads) k_m2l_build(BuildArgs a, int k, const double* cheb, const double* Rt,
                                                        double* far0) {
    extern __shared__ double msm[];  // Kc (r0 x r0), tmp (r0 x r0)
    const int b = blockIdx.x, j = blockIdx.y;
    const int side = 1 << k;
    const Cell cb = cell_of(b, side, a.dim);
    const Cell cq = region_cell(cb, j, a.dim);
    const int r0 = a.r0, p = a.p;
    const int nreg = nregion(a.dim);
    double* out = far0 + ((int64_t)b * nreg + j) * r0 * r0;
    if (!cell_in(cq, side) || cheb_dist(cq, cb) <= 1) return;
    const int q = cell_index(cq, side);
    const double h = a.L / side;
    double* Kc = msm;
    double* tmp = msm + r0 * r0;
    const bool d3 = a.dim == 3;
    for (int t = threadIdx.x; t < r0 * r0; t += blockDim.x) {
        int m = t / r0, l = t - m * r0;
        double ax = a.x0 + (cb.x + 0.5 * (cheb[m % p] + 1.0)) * h, ay = a.y0 + (cb.y + 0.5 * (cheb[(m / p) % p] + 1.0)) * h;
        double cx = a.x0 + (cq.x + 0.5 * (cheb[l % p] + 1.0)) * h, cy = a.y0 + (cq.y + 0.5 * (cheb[(l / p) % p] + 1.0)) * h;
        double az = d3 ? a.z0 + (cb.z + 0.5 * (cheb[m / (p * p)] + 1.0)) * h : 0.0;
        double cz = d3 ? a.z0 + (cq.z + 0.5 * (cheb[l / (p * p)] + 1.0)) * h : 0.0;
        Kc[t] = kernel_eval(a.kernel, a.kparam0, ax, ay, az, cx, cy, cz);
    }
    __syncthreads();
    const double* Rb = Rt + (int64_t)b * r0 * r0;
    const double* Rq = Rt + (int64_t)q * r0 * r0;
    for (int t = threadIdx.x; t < r0 * r0; t += blockDim.x) {  // tmp = Rb Kc
        int i = t / r0, l = t - i * r0;
        double s = 0.0;
        for (int m = 0; m < r0; ++m) s += Rb[(size_t)i * r0 + m] * Kc[(size_t)m * r0 + l];
        tmp[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < r0 * r0; t += blockDim.x) {  // out = tmp Rq^T
        int i = t / r0, jj = t - i * r0;
        double s = 0.0;
        for (int l = 0; l < r0; ++l) s += tmp[(size_t)i * r0 + l] * Rq[(size_t)jj * r0 + l];
        out[t] = s;
    }
}

void launch_m2l_build(const BuildArgs& a, int k, const double* cheb, const double* Rt, double* far0,
                      cudaStream_t st) {
    size_t smem = 2 * (size_t)a.r0 * a.r0 * sizeof(double);
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        cudaFuncSetAttribute(k_m2l_build, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr.store(true);
    }
    k_m2l_build<<<dim3(1u << (a.dim * k), nregion(a.dim)), kThreads, smem, st>>>(a, k, cheb, Rt, far0);
    count_launches(1);
}

// leaf P2P blocks and the matrix scale s_A (largest column norm of the diagonal blocks)
__global__ void __launch_bounds__(kThreads) k_p2p_build(BuildArgs a, const double* px, const double* py,
                                                        const double* pz, const int64_t* leaf_start,
                                                        const int* leaf_count, const int64_t* p2p_off, double* p2p,
                                                        unsigned long long* sA_bits) {
    const int b = blockIdx.x, d = blockIdx.y;
    const int side = 1 << a.depth, nd = ndirs(a.dim);
    const Cell cq = cell_dir(cell_of(b, side, a.dim), d, a.dim);
    if (!cell_in(cq, side)) return;
    const int q = cell_index(cq, side);
    const int nb_ = leaf_count[b], nq = leaf_count[q];
    const int64_t sb = leaf_start[b], sq = leaf_start[q];
    double* out = p2p + p2p_off[(int64_t)b * nd + d];
    for (int t = threadIdx.x; t < nb_ * nq; t += blockDim.x) {
        int i = t / nq, j = t - i * nq;
        double v = (b == q && i == j) ? a.diag
                                      : kernel_eval(a.kernel, a.kparam0, px[sb + i], py[sb + i], pz[sb + i], px[sq + j],
                                                    py[sq + j], pz[sq + j]);
        out[t] = v;
    }
    if (d != nd / 2) return;
    __syncthreads();
    double mx = 0.0;
    for (int j = threadIdx.x; j < nq; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < nb_; ++i) s += out[(size_t)i * nq + j] * out[(size_t)i * nq + j];
        mx = fmax(mx, sqrt(s));
    }
    if (mx > 0.0) atomicMax(sA_bits, (unsigned long long)__double_as_longlong(mx));
}

void launch_p2p_build(const BuildArgs& a, const double* px, const double* py, const double* pz,
                      const int64_t* leaf_start, const int* leaf_count, const int64_t* p2p_off, double* p2p,
                      double* sA_bits, cudaStream_t st) {
    k_p2p_build<<<dim3(1u << (a.dim * a.depth), ndirs(a.dim)), kThreads, 0, st>>>(
        a, px, py, pz, leaf_start, leaf_count, p2p_off, p2p, reinterpret_cast<unsigned long long*>(sA_bits));
    count_launches(1);
}

// ---------------------------------------------------------------------------------------------
// FMM matvec y = A~ x (Table "table_FMM_operators"), element type T: FP64 for the residuals of the
// refinement, double-float (operators split once into double-float copies) for the inner Krylov
// steps of the mixed-precision solve. Vectors outside are FP64; the permutation kernels convert.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_mv_permute_in(const double* x, int64_t ld, int64_t N, int nrhs, const int64_t* perm, T* xt) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * nrhs) return;
    int64_t i = t / nrhs;
    int j = (int)(t - i * nrhs);
    xt[t] = (T)x[perm[i] + (int64_t)j * ld];
}
template <typename T>
void launch_mv_permute_in(const double* x, int64_t ld, int64_t N, int nrhs, const int64_t* perm, T* xt,
                          cudaStream_t st) {
    k_mv_permute_in<T><<<(unsigned)((N * nrhs + 255) / 256), 256, 0, st>>>(x, ld, N, nrhs, perm, xt); count_launches(1);
}

template <typename T>
__global__ void k_mv_permute_out(const T* yt, int64_t N, int nrhs, const int64_t* perm, double* y, int64_t ld) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * nrhs) return;
    int64_t i = t / nrhs;
    int j = (int)(t - i * nrhs);
    y[perm[i] + (int64_t)j * ld] = (double)yt[t];
}
template <typename T>
void launch_mv_permute_out(const T* yt, int64_t N, int nrhs, const int64_t* perm, double* y, int64_t ld,
                           cudaStream_t st) {
    k_mv_permute_out<T><<<(unsigned)((N * nrhs + 255) / 256), 256, 0, st>>>(yt, N, nrhs, perm, y, ld); count_launches(1);
}

// P2M: y_b = W0_b^T x_b   (y layout [box][r0][nrhs])
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mv_leaf_up(const T* W0, const int64_t* leaf_start,
                                                         const int* leaf_count, int r0, const T* xt, T* y,
                                                         int nrhs) {
    __shared__ T sm[gemm_smem<T>::value];
    const int b = blockIdx.x;
    const int64_t s0 = leaf_start[b];
    const int n = leaf_count[b];
    const T* W = W0 + s0 * r0;
    const T* xb = xt + s0 * nrhs;
    T* yb = y + (int64_t)b * r0 * nrhs;
    cta_gemm<T>(
        r0, nrhs, n, [&](int i, int k) { return W[(size_t)k * r0 + i]; },
        [&](int k, int j) { return xb[(size_t)k * nrhs + j]; },
        [&](int i, int j, T v) { yb[(size_t)i * nrhs + j] = v; }, sm);
}
template <typename T>
void launch_mv_leaf_up(int dim, int depth, const T* W0, const int64_t* leaf_start, const int* leaf_count, int r0,
                       const T* xt, T* y, int nrhs, cudaStream_t st) {
    k_mv_leaf_up<T><<<1u << (dim * depth), kThreads, 0, st>>>(W0, leaf_start, leaf_count, r0, xt, y, nrhs);
    count_launches(1);
}

// M2M: y_P = W0_P^T [y_c]  (W0_P rows c*r0 + t, 2^d children)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mv_up(int dim, int k, const T* W0, int r0, const T* ychild, T* y,
                                                    int nrhs) {
    __shared__ T sm[gemm_smem<T>::value];
    const int b = blockIdx.x;
    const int side = 1 << k, cs = side << 1, nk = 1 << dim;
    const Cell cb = cell_of(b, side, dim);
    const T* W = W0 + (int64_t)b * nk * r0 * r0;
    T* yb = y + (int64_t)b * r0 * nrhs;
    cta_gemm<T>(
        r0, nrhs, nk * r0, [&](int i, int kk) { return W[(size_t)kk * r0 + i]; },
        [&](int kk, int j) {
            int c = kk / r0, t = kk - c * r0;
            int cg = cell_index(child_cell(cb, c), cs);
            return ychild[((int64_t)cg * r0 + t) * nrhs + j];
        },
        [&](int i, int j, T v) { yb[(size_t)i * nrhs + j] = v; }, sm);
}
template <typename T>
void launch_mv_up(int dim, int k, const T* W0, int r0, const T* ychild, T* y, int nrhs, cudaStream_t st) {
    k_mv_up<T><<<1u << (dim * k), kThreads, 0, st>>>(dim, k, W0, r0, ychild, y, nrhs);
    count_launches(1);
}

// M2L: z_b = sum_{q in I_b} M2L_bq y_q
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mv_m2l(int dim, int k, const T* far0, int r0, const T* y, T* z,
                                                     int nrhs) {
    __shared__ T sm[gemm_smem<T>::value];
    const int b = blockIdx.x;
    const int side = 1 << k, nreg = nregion(dim);
    const Cell cb = cell_of(b, side, dim);
    T* zb = z + (int64_t)b * r0 * nrhs;
    for (int t = threadIdx.x; t < r0 * nrhs; t += blockDim.x) zb[t] = (T)0;
    __syncthreads();
    for (int j = 0; j < nreg; ++j) {
        const Cell cq = region_cell(cb, j, dim);
        if (!cell_in(cq, side) || cheb_dist(cq, cb) <= 1) continue;
        const int q = cell_index(cq, side);
        const T* M = far0 + ((int64_t)b * nreg + j) * r0 * r0;
        const T* yq = y + (int64_t)q * r0 * nrhs;
        cta_gemm<T>(
            r0, nrhs, r0, [&](int i, int kk) { return M[(size_t)i * r0 + kk]; },
            [&](int kk, int jj) { return yq[(size_t)kk * nrhs + jj]; },
            [&](int i, int jj, T v) { zb[(size_t)i * nrhs + jj] += v; }, sm);
        __syncthreads();
    }
}
template <typename T>
void launch_mv_m2l(int dim, int k, const T* far0, int r0, const T* y, T* z, int nrhs, cudaStream_t st) {
    k_mv_m2l<T><<<1u << (dim * k), kThreads, 0, st>>>(dim, k, far0, r0, y, z, nrhs);
    count_launches(1);
}

// L2L: z_c += W0_P[rows of c] z_P, one block per child box c at level k+1
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mv_down(int dim, int k, const T* W0, int r0, const T* z, T* zchild,
                                                      int nrhs) {
    __shared__ T sm[gemm_smem<T>::value];
    const int cgi = blockIdx.x;
    const int cs = 2 << k, nk = 1 << dim;
    const Cell cc = cell_of(cgi, cs, dim);
    const int P = cell_index(Cell{cc.x >> 1, cc.y >> 1, cc.z >> 1}, cs >> 1);
    const int c = (cc.x & 1) + 2 * (cc.y & 1) + 4 * (cc.z & 1);
    const T* W = W0 + ((int64_t)P * nk + c) * r0 * r0;
    const T* zP = z + (int64_t)P * r0 * nrhs;
    T* zc = zchild + (int64_t)cgi * r0 * nrhs;
    cta_gemm<T>(
        r0, nrhs, r0, [&](int i, int kk) { return W[(size_t)i * r0 + kk]; },
        [&](int kk, int j) { return zP[(size_t)kk * nrhs + j]; },
        [&](int i, int j, T v) { zc[(size_t)i * nrhs + j] += v; }, sm);
}
template <typename T>
void launch_mv_down(int dim, int k, const T* W0, int r0, const T* z, T* zchild, int nrhs, cudaStream_t st) {
    k_mv_down<T><<<1u << (dim * (k + 1)), kThreads, 0, st>>>(dim, k, W0, r0, z, zchild, nrhs);
    count_launches(1);
}

// L2P + P2P: out_b = W0_b z_b + sum_{q in N_b} P2P_bq x_q
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mv_leaf_down(int dim, int depth, const T* W0, const int64_t* leaf_start,
                                                           const int* leaf_count, int r0, const T* z, const T* xt,
                                                           const int64_t* p2p_off, const T* p2p, T* out, int nrhs) {
    __shared__ T sm[gemm_smem<T>::value];
    const int b = blockIdx.x;
    const int side = 1 << depth, nd = ndirs(dim);
    const Cell cb = cell_of(b, side, dim);
    const int64_t s0 = leaf_start[b];
    const int n = leaf_count[b];
    const T* W = W0 + s0 * r0;
    const T* zb = z + (int64_t)b * r0 * nrhs;
    T* ob = out + s0 * nrhs;
    cta_gemm<T>(
        n, nrhs, r0, [&](int i, int kk) { return W[(size_t)i * r0 + kk]; },
        [&](int kk, int j) { return zb[(size_t)kk * nrhs + j]; },
        [&](int i, int j, T v) { ob[(size_t)i * nrhs + j] = v; }, sm);
    __syncthreads();
    for (int d = 0; d < nd; ++d) {
        const Cell cq = cell_dir(cb, d, dim);
        if (!cell_in(cq, side)) continue;
        const int q = cell_index(cq, side);
        const int nq = leaf_count[q];
        const T* B = p2p + p2p_off[(int64_t)b * nd + d];
        const T* xq = xt + leaf_start[q] * nrhs;
        cta_gemm<T>(
            n, nrhs, nq, [&](int i, int kk) { return B[(size_t)i * nq + kk]; },
            [&](int kk, int j) { return xq[(size_t)kk * nrhs + j]; },
            [&](int i, int j, T v) { ob[(size_t)i * nrhs + j] += v; }, sm);
        __syncthreads();
    }
}
template <typename T>
void launch_mv_leaf_down(int dim, int depth, const T* W0, const int64_t* leaf_start, const int* leaf_count, int r0,
                         const T* z, const T* xt, const int64_t* p2p_off, const T* p2p, T* out, int nrhs,
                         cudaStream_t st) {
    k_mv_leaf_down<T><<<1u << (dim * depth), kThreads, 0, st>>>(dim, depth, W0, leaf_start, leaf_count, r0, z, xt,
                                                                p2p_off, p2p, out, nrhs);
    count_launches(1);
}

// split of an FP64 array into double-float pairs
// A streaming copy (each element read and written once, 16 bytes per element pair): with both
// pointers 16-byte aligned, each thread moves pairs as one 16-byte load and one 16-byte store, four
// pairs in flight per loop step, with evict-first hints (the copies are read again only after
// gigabytes of other traffic); otherwise one element at a time.
__device__ __forceinline__ float4 split_pair(double2 v) {
    const dfl x(v.x), y(v.y);
    return make_float4(x.hi, x.lo, y.hi, y.lo);
}
__global__ void k_split_dfl(const double* __restrict__ a, dfl* __restrict__ b, int64_t n, int vec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!vec) {
        for (int64_t i = t; i < n; i += stride) b[i] = dfl(a[i]);
        return;
    }
    const int64_t n2 = n >> 1;
    const double2* a2 = reinterpret_cast<const double2*>(a);
    float4* b4 = reinterpret_cast<float4*>(b);
    int64_t i = t;
    for (; i + 3 * stride < n2; i += 4 * stride) {
        const double2 v0 = __ldcs(a2 + i), v1 = __ldcs(a2 + i + stride);
        const double2 v2 = __ldcs(a2 + i + 2 * stride), v3 = __ldcs(a2 + i + 3 * stride);
        __stcs(b4 + i, split_pair(v0));
        __stcs(b4 + i + stride, split_pair(v1));
        __stcs(b4 + i + 2 * stride, split_pair(v2));
        __stcs(b4 + i + 3 * stride, split_pair(v3));
    }
    for (; i < n2; i += stride) __stcs(b4 + i, split_pair(__ldcs(a2 + i)));
    if (t == 0 && (n & 1)) b[n - 1] = dfl(a[n - 1]);
}
void launch_split_dfl(const double* a, dfl* b, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    const int vec = (((uintptr_t)a | (uintptr_t)b) & 15u) == 0;
    const int64_t work = vec ? (n + 1) / 2 : n;
    k_split_dfl<<<(unsigned)std::min<int64_t>((work + 255) / 256, 152 * 8), 256, 0, st>>>(a, b, n, vec);
    count_launches(1);
}

#define IFMM_MV_INSTANTIATE(T)                                                                                    \
    template void launch_mv_permute_in<T>(const double*, int64_t, int64_t, int, const int64_t*, T*, cudaStream_t); \
    template void launch_mv_permute_out<T>(const T*, int64_t, int, const int64_t*, double*, int64_t, cudaStream_t); \
    template void launch_mv_leaf_up<T>(int, int, const T*, const int64_t*, const int*, int, const T*, T*, int,    \
                                       cudaStream_t);                                                            \
    template void launch_mv_up<T>(int, int, const T*, int, const T*, T*, int, cudaStream_t);                      \
    template void launch_mv_m2l<T>(int, int, const T*, int, const T*, T*, int, cudaStream_t);                     \
    template void launch_mv_down<T>(int, int, const T*, int, const T*, T*, int, cudaStream_t);                    \
    template void launch_mv_leaf_down<T>(int, int, const T*, const int64_t*, const int*, int, const T*, const T*, \
                                         const int64_t*, const T*, T*, int, cudaStream_t);
IFMM_MV_INSTANTIATE(double)
IFMM_MV_INSTANTIATE(dfl)
#undef IFMM_MV_INSTANTIATE

// The refinement's reductions over N run in two steps so that they give the same bits run after
// run: each block writes its partial sum to part[block * nout + output] (no atomics), then
// k_sum_partials adds the partials of every output in block order.
__global__ void k_sum_partials(const double* part, int nblk, int nout, double* out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    double s = 0.0;
    for (int x = 0; x < nblk; ++x) s += part[(size_t)x * nout + o];
    out[o] += s;
}
static void sum_partials(const double* part, int nblk, int nout, double* out, cudaStream_t st) {
    k_sum_partials<<<(nout + 255) / 256, 256, 0, st>>>(part, nblk, nout, out);
    count_launches(1);
}
static int vec_blocks(int64_t N) { return (int)std::min<int64_t>((N + 255) / 256, 1024); }
static int dot_blocks(int64_t N) { return (int)((N + 4095) / 4096); }
size_t reduction_scratch_doubles(int64_t N, int nrhs, int cnt) {
    return std::max((size_t)dot_blocks(N) * (size_t)std::max(cnt, 1), (size_t)vec_blocks(N) * 2) * (size_t)nrhs;
}

// x += d (d with leading dimension N); nrm[2j] += ||d_j||^2, nrm[2j+1] += ||x_j||^2 (x after the update)
__global__ void k_axpy_norms(double* x, const double* d, int64_t N, int nrhs, int64_t ld, double* part) {
    __shared__ double red[32];
    const int j = blockIdx.y;
    double sd = 0.0, sx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double dv = d[i + j * N];
        double xv = x[i + j * ld] + dv;
        x[i + j * ld] = xv;
        sd += dv * dv;
        sx += xv * xv;
    }
    sd = block_sum(sd, red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 2 * nrhs + 2 * j] = sd;
    sx = block_sum(sx, red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 2 * nrhs + 2 * j + 1] = sx;
}
void launch_axpy_norms(double* x, const double* d, int64_t N, int nrhs, int64_t ld, double* nrm, double* part,
                       cudaStream_t st) {
    const int gx = vec_blocks(N);
    k_axpy_norms<<<dim3(gx, nrhs), 256, 0, st>>>(x, d, N, nrhs, ld, part); count_launches(1);
    sum_partials(part, gx, 2 * nrhs, nrm, st);
}

// r = b - ax; nrm[2j] += ||r_j||^2, nrm[2j+1] += ||b_j||^2
__global__ void k_residual(const double* b, const double* ax, double* r, int64_t N, int nrhs, int64_t ld, double* part) {
    __shared__ double red[32];
    const int j = blockIdx.y;
    double sr = 0.0, sb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double bv = b[i + j * ld];
        double rv = bv - ax[i + j * N];
        r[i + j * N] = rv;
        sr += rv * rv;
        sb += bv * bv;
    }
    sr = block_sum(sr, red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 2 * nrhs + 2 * j] = sr;
    sb = block_sum(sb, red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 2 * nrhs + 2 * j + 1] = sb;
}
void launch_residual(const double* b, const double* ax, double* r, int64_t N, int nrhs, int64_t ld, double* nrm,
                     double* part, cudaStream_t st) {
    const int gx = vec_blocks(N);
    k_residual<<<dim3(gx, nrhs), 256, 0, st>>>(b, ax, r, N, nrhs, ld, part); count_launches(1);
    sum_partials(part, gx, 2 * nrhs, nrm, st);
}

// ---------------------------------------------------------------------------------------------
// FP64 Krylov vector kernels for the refinement (all nrhs columns at once, column-major, ld N)
// ---------------------------------------------------------------------------------------------
// out[i * nrhs + c] += sum_n V_i[n, c] w[n, c] for i < cnt (V_i = V + i * N * nrhs)
__global__ void __launch_bounds__(256) k_krylov_dots(const double* V, int cnt, const double* w, int64_t N, int nrhs,
                                                     double* part) {
    __shared__ double red[32];
    constexpr int PER = 16;
    const int c = blockIdx.y;
    const int64_t n0 = (int64_t)blockIdx.x * 256 * PER;
    double wv[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        int64_t n = n0 + threadIdx.x + 256 * t;
        wv[t] = n < N ? w[n + (int64_t)c * N] : 0.0;
    }
    for (int i = 0; i < cnt; ++i) {
        const double* v = V + (int64_t)i * N * nrhs + (int64_t)c * N;
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            int64_t n = n0 + threadIdx.x + 256 * t;
            if (n < N) s += v[n] * wv[t];
        }
        s = block_sum(s, red);
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * cnt * nrhs + (size_t)i * nrhs + c] = s;
    }
}
void launch_krylov_dots(const double* V, int cnt, const double* w, int64_t N, int nrhs, double* out, double* part,
                        cudaStream_t st) {
    const int gx = dot_blocks(N);
    k_krylov_dots<<<dim3((unsigned)gx, nrhs), 256, 0, st>>>(V, cnt, w, N, nrhs, part);
    count_launches(1);
    sum_partials(part, gx, cnt * nrhs, out, st);
}

// y[n + c * ldy] += sum_i coef[i * nrhs + c] V_i[n, c]
__global__ void k_krylov_lincomb(const double* V, int cnt, const double* coef, double* y, int64_t ldy, int64_t N,
                                 int nrhs) {
    const int c = blockIdx.y;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < cnt; ++i) acc += coef[i * nrhs + c] * V[(int64_t)i * N * nrhs + (int64_t)c * N + n];
        y[n + (int64_t)c * ldy] += acc;
    }
}
void launch_krylov_lincomb(const double* V, int cnt, const double* coef, double* y, int64_t ldy, int64_t N, int nrhs,
                           cudaStream_t st) {
    int gx = (int)std::min<int64_t>((N + 255) / 256, 2048);
    k_krylov_lincomb<<<dim3(gx, nrhs), 256, 0, st>>>(V, cnt, coef, y, ldy, N, nrhs);
    count_launches(1);
}

// out[c] += ||y[:, c]||^2 ; then optionally y[:, c] *= scale[c]
__global__ void k_colnorm2(const double* y, int64_t ldy, int64_t N, int nrhs, double* part) {
    __shared__ double red[32];
    const int c = blockIdx.y;
    double s = 0.0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        double v = y[n + (int64_t)c * ldy];
        s += v * v;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * nrhs + c] = s;
}
void launch_colnorm2(const double* y, int64_t ldy, int64_t N, int nrhs, double* out, double* part, cudaStream_t st) {
    const int gx = vec_blocks(N);
    k_colnorm2<<<dim3(gx, nrhs), 256, 0, st>>>(y, ldy, N, nrhs, part);
    count_launches(1);
    sum_partials(part, gx, nrhs, out, st);
}

__global__ void k_colscale(double* y, int64_t ldy, int64_t N, const double* scale) {
    const int c = blockIdx.y;
    const double s = scale[c];
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        y[n + (int64_t)c * ldy] *= s;
}
void launch_colscale(double* y, int64_t ldy, int64_t N, int nrhs, const double* scale, cudaStream_t st) {
    int gx = (int)std::min<int64_t>((N + 255) / 256, 2048);
    k_colscale<<<dim3(gx, nrhs), 256, 0, st>>>(y, ldy, N, scale);
    count_launches(1);
}

}  // namespace ifmm
