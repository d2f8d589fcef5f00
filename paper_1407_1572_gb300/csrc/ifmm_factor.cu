// ifmm_factor.cu -- elimination (Algorithm 1) and replay (Algorithm 2) kernels, sm_103a.
//
// One colour of one level is eliminated by five launches over the boxes of that colour
// (colour = (ix mod 3) + 3 (iy mod 3) (+ 9 (iz mod 3) in 3D): boxes of one colour are at Chebyshev
// distance >= 3, so their neighbourhoods N_e, and every block they touch, are disjoint). A launch's
// blockIdx.y is a neighbour direction (3^d of them) or an ordered pair of directions (9^d):
//   k_pivot    form Piv_e = [[P2P_ee, L2P_ee], [P2M_ee, 0]] (rows P2P(e,k), P2M(e,k), columns
//              x_e, z_e) and invert it in FP64 (Gauss-Jordan, partial pivoting);
//   k_panel    X = Piv_e^{-1} [B; 0] for every neighbour column block (B = row P2P_e at the
//              neighbour's active unknown) and for y_e; save the B and C panels for the solve;
//   k_schur    Schur complement A[rho, gamma] -= C_rho X_gamma over the neighbour pairs: dense
//              update of neighbour blocks, well-separated fill written out for compression;
//   k_compress per uneliminated neighbour q: extend its basis W_q by the directions of its
//              well-separated fill that W_q misses (pivoted Gram-Schmidt with threshold);
//   k_redirect write each well-separated fill through the bases into M2L_pq
//              (Algorithm 1: P2P_pq = L2P_pp M2L_pq P2M_qq, P2L_pq = M2L_pq P2M_qq,
//              M2P_pq = L2P_pp M2L_pq).
// T is the storage type of blocks, bases and panels (double, or float in the mixed form).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cooperative_groups.h>

#include "ifmm_common.cuh"
#include "ifmm_internal.h"
#include "ifmm_tc.cuh"

namespace ifmm {

// per host thread, so that handles factored or solved concurrently by different threads each count
// their own launches
static thread_local long long g_launches = 0;
void count_launches(int n) { g_launches += n; }
long long launches_so_far() { return g_launches; }
int num_sms();

// largest cluster of blocks one compression may be spread over (1: one block per compression)
static std::atomic<int> compress_cluster_max{16};
int set_compress_cluster(int c) {
    if (c != 1 && c != 2 && c != 4 && c != 8 && c != 16) return -1;
    compress_cluster_max.store(c);
    return 0;
}

template <typename T> struct AccOf { using type = double; };
template <> struct AccOf<float> { using type = float; };
template <> struct AccOf<dfl> { using type = dfl; };

// (2D grid test of the tensor-core replay kernels, which serve quadtrees only)
IFMM_DEVINL bool in_grid(int x, int y, int side) { return x >= 0 && y >= 0 && x < side && y < side; }

template <typename T>
IFMM_DEVINL T* block_at(const LevelView<T>& L, int p, int q, int& ld) {
    const int j = region_index(cell_of(p, L.side, L.dim), cell_of(q, L.side, L.dim), L.dim);
    int64_t o = L.boff[(int64_t)p * L.nreg + j];
    ld = L.bld[(int64_t)p * L.nreg + j];
    return o < 0 ? nullptr : L.blk + o;
}

// offset of the fill of the ordered direction pair (da, db) of box e
template <typename T>
IFMM_DEVINL int64_t fill_off(const LevelView<T>& L, int e, int da, int db) {
    return L.fsoff[((int64_t)e * L.nd + da) * L.nd + db];
}

// column offset inside X of the block of neighbour direction dsel (dsel == ctr: the y_e block)
template <typename T>
IFMM_DEVINL int xcol_offset(const LevelView<T>& L, Cell ce, int dsel) {
    int off = 0;
    for (int d = 0; d < L.nd; ++d) {
        if (d == L.ctr) continue;
        if (d == dsel) return off;
        const Cell cq = cell_dir(ce, d, L.dim);
        if (cell_in(cq, L.side)) off += L.n[cell_index(cq, L.side)];
    }
    return off;
}

// element (i, j) of the well-separated fill F_ab (wa x wb) of the eliminated box e, ordered
// directions da, db. For a symmetric kernel only the pair with da < db is stored (F_ba = F_ab^T).
template <typename T>
IFMM_DEVINL T fill_at(const LevelView<T>& L, int e, int da, int db, int wa, int wb, int i, int j) {
    if (!L.symmetric || da < db) return L.Fs[fill_off(L, e, da, db) + (size_t)i * wb + j];
    return L.Fs[fill_off(L, e, db, da) + (size_t)j * wa + i];
}

// active width of box b while eliminating colour c: r_b once eliminated, n_b before
template <typename T>
IFMM_DEVINL int active_width(const LevelView<T>& L, int b, int colour) {
    return cell_colour(cell_of(b, L.side, L.dim)) < colour ? L.r[b] : L.n[b];
}

// ---------------------------------------------------------------------------------------------
// k_pivot: Piv_e^{-1} in FP64
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pivot(LevelView<T> L0, BoxList<T> bl, int smax, int use_smem) {
    const LevelView<T>& L = bl.view(L0, blockIdx.x);
    extern __shared__ double dsm[];
    __shared__ double vred[32];
    __shared__ int ired[32];
    const int e = bl.box(blockIdx.x);
    const int n = L.n[e], r = L.r[e], s = n + r;
    if (s == 0) return;
    double* col = dsm;
    int* perm = reinterpret_cast<int*>(dsm + smax);
    double* A = use_smem ? dsm + smax + (smax + 1) / 2 : L.pws + L.psoff[e];
    int ldp;
    const T* Pee = block_at(L, e, e, ldp);
    const T* We = L.W + L.voff[e] * L.RC;
    const int RC = L.RC;
    // balancing a = largest column norm of P2P_ee: the block is inverted as
    // Piv_s = [[P2P_ee, a W], [a W^T, 0]] and Piv^{-1} = S Piv_s^{-1} S, S = diag(I_n, a I_r)
    double cmax = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double c = 0.0;
        for (int i = 0; i < n; ++i) {
            double v = (double)Pee[(size_t)i * ldp + j];
            c += v * v;
        }
        cmax = fmax(cmax, sqrt(c));
    }
    double alpha = block_max(cmax, vred);
    if (!(alpha > 0.0)) alpha = 1.0;
    for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
        int i = t / s, j = t - i * s;
        double v;
        if (i < n && j < n) v = (double)Pee[(size_t)i * ldp + j];
        else if (i < n) v = alpha * (double)We[(size_t)i * RC + (j - n)];
        else if (j < n) v = alpha * (double)We[(size_t)j * RC + (i - n)];
        else v = 0.0;
        A[(size_t)i * s + j] = v;
    }
    __syncthreads();
    bool ok = cta_gauss_jordan(A, s, s, perm, col, vred, ired);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(L.status, DEV_ERR_SINGULAR);
        return;
    }
    T* Pi = L.Pi + L.pioff[e];
    const int ld = L.pild[e];
    for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
        int i = t / s, j = t - i * s;
        double sc = (i >= n ? alpha : 1.0) * (j >= n ? alpha : 1.0);
        Pi[(size_t)i * ld + j] = (T)(sc * A[(size_t)i * s + j]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&L.counters[2], 2.0 * s * (double)s * s);
        atomicAdd(&L.counters[3], 2.0 * s * (double)s * s);
    }
}

// The best (largest value, ties to the lowest index; index < 0: no candidate) of the candidates
// (*val, *idx) that the C blocks of a cluster hold in shared memory: lane j of every warp reads block
// j's, the warp reduces them, and lane 0's result is broadcast, so that every thread of every block
// takes the same choice (the comparisons are the same in all of them, whatever the values).
template <class CL>
IFMM_DEVINL int cluster_pick(CL& cl, double* val, int* idx, int C, double* vout) {
    const int lane = (int)threadIdx.x & 31;
    double v = -1.0;
    int i = -1;
    if (lane < C) {
        v = *cl.map_shared_rank(val, lane);
        i = *cl.map_shared_rank(idx, lane);
    }
    for (int o = C >> 1; o > 0; o >>= 1) {   // (C a power of two: lanes 0 .. C-1 combine)
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (oi >= 0 && (i < 0 || ov > v || (ov == v && oi < i))) { v = ov; i = oi; }
    }
    *vout = __shfl_sync(0xffffffffu, v, 0);
    return __shfl_sync(0xffffffffu, i, 0);
}

// ---------------------------------------------------------------------------------------------
// k_pivot_cluster: the same balanced FP64 Gauss-Jordan inversion for large pivot blocks, spread
// over a cluster of C blocks (one box per cluster). Row i lives in block i mod C (local row
// i / C). Row interchanges are implicit: at step k the pivot is the unused row p_k with the
// largest |A[p_k][k]| (ties to the lowest row); in exchange form the tableau then holds
// A^{-1}[k][p_j] = R[p_k][j], applied when Pi is written. Per step: candidates are exchanged
// through distributed shared memory (cluster barrier), the owner scales the pivot row, every
// block copies it (cluster barrier) and updates its own rows. Every block runs the same
// number of cluster barriers (the pivot choice is computed identically in all of them).
// Shared memory: slab (rows_loc x s, or in the box's global FP64 workspace when slab_global),
// prow (s), fcol (2 x rows_loc), perm (s), used (rows_loc). Cluster sizes up to 16 (16: non-portable).
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pivot_cluster(LevelView<T> L0, BoxList<T> bl, int C, int smax,
                                                            int slab_global) {
    // pivot blocks are inverted in FP64 in every precision mode: they are the ill-conditioned part
    // of the elimination (balanced condition numbers up to 5e7 on uniform clouds, worse on
    // clustered ones), where a 48-bit double-float inversion broke GMRES on Gaussian-blob systems
    using S = double;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double dsm[];
    __shared__ double vred[32];
    __shared__ double s_cval;
    __shared__ int s_cidx;
    __shared__ double s_alpha;
    const int c = (int)cl.block_rank();
    const LevelView<T>& L = bl.view(L0, blockIdx.x / C);
    const int e = bl.box(blockIdx.x / C);
    const int n = L.n[e], r = L.r[e], s = n + r;
    const int rows_max = (smax + C - 1) / C;
    double* base = slab_global ? dsm : dsm + (size_t)rows_max * smax;
    S* prow = reinterpret_cast<S*>(base);             // smax
    S* fcol = prow + smax;                            // 2 x rows_max
    int* perm = reinterpret_cast<int*>(fcol + 2 * rows_max);  // smax
    int* used = perm + smax;                          // rows_max
    const int rows_loc = s > c ? (s - c + C - 1) / C : 0;
    // local row tl of this block is global row c + tl C: in shared memory (slab_global = 0) at
    // dsm + tl s, in global memory at row c + tl C of the box's s x s workspace
    S* slab = reinterpret_cast<S*>(slab_global ? L.pws + L.psoff[e] + (size_t)c * s : dsm);
    const size_t sstride = slab_global ? (size_t)C * s : (size_t)s;
    int ldp;
    const T* Pee = block_at(L, e, e, ldp);
    const T* We = L.W + L.voff[e] * L.RC;
    const int RC = L.RC;
    // balancing a = largest column norm of P2P_ee (same in every block of the cluster)
    double cmax = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            double v = (double)Pee[(size_t)i * ldp + j];
            acc += v * v;
        }
        cmax = fmax(cmax, sqrt(acc));
    }
    double alpha = block_max(cmax, vred);
    if (!(alpha > 0.0)) alpha = 1.0;
    if (threadIdx.x == 0) s_alpha = alpha;
    // element t = tl s + j of the local rows, walked in steps of the block size without a division
    // per element: (tl, j) advances by (dr, dc) with blockDim = dr s + dc
    const int sd = s > 0 ? s : 1;   // an empty box (s = 0) has no local rows
    const int dr = (int)blockDim.x / sd, dc = (int)blockDim.x - dr * sd;
    const int tl0 = (int)threadIdx.x / sd, j0 = (int)threadIdx.x - tl0 * sd;
    for (int tl = tl0, j = j0; tl < rows_loc;) {
        const int i = c + tl * C;
        double v;
        if (i < n && j < n) v = (double)Pee[(size_t)i * ldp + j];
        else if (i < n) v = alpha * (double)We[(size_t)i * RC + (j - n)];
        else if (j < n) v = alpha * (double)We[(size_t)j * RC + (i - n)];
        else v = 0.0;
        slab[(size_t)tl * sstride + j] = S(v);
        tl += dr;
        j += dc;
        if (j >= s) { j -= s; ++tl; }
    }
    __syncthreads();   // the slab's rows are written by other threads than those that read column 0
    // column k of the local rows before step k: fcol[k & 1] (written by step k - 1, for every row:
    // the pivot row as it is scaled, the others as they are updated), so that neither the pivot
    // search nor the update reads a column of the slab with a stride of s
    for (int t = threadIdx.x; t < rows_loc; t += blockDim.x) {
        used[t] = 0;
        fcol[t] = slab[(size_t)t * sstride];
    }
    __syncthreads();
    for (int k = 0; k < s; ++k) {
        const S* fc = fcol + (k & 1) * rows_max;
        S* fn = fcol + ((k + 1) & 1) * rows_max;
        // local candidate among unused rows (one warp; ties to the lowest row)
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = -1;
            for (int tl = threadIdx.x; tl < rows_loc; tl += 32) {
                if (used[tl]) continue;
                const double v = sc_mag(fc[tl]);
                const int gi = c + tl * C;
                if (bi < 0 || v > best || (v == best && gi < bi)) { best = v; bi = gi; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (oi >= 0 && (bi < 0 || ov > best || (ov == best && oi < bi))) { best = ov; bi = oi; }
            }
            if (threadIdx.x == 0) { s_cval = best; s_cidx = bi; }
        }
        cl.sync();
        // global pivot: identical choice in every block
        double gv;
        const int p = cluster_pick(cl, &s_cval, &s_cidx, C, &gv);
        if (p < 0 || !(gv > 0.0) || !isfinite(gv)) {
            if (threadIdx.x == 0 && c == 0) atomicOr(L.status, DEV_ERR_SINGULAR);
            cl.sync();  // every block leaves at the same step, after all candidate reads
            return;
        }
        const int owner = p % C, tp = p / C;
        if (threadIdx.x == 0) perm[k] = p;
        if (c == owner) {
            // the pivot A[p][k] is fc[tp], so no barrier separates its read from the row's overwrite
            const S d = S(1.0 / (double)fc[tp]);
            for (int j = threadIdx.x; j < s; j += blockDim.x) {
                const S v = (j == k) ? d : sc_mul(slab[(size_t)tp * sstride + j], d);
                slab[(size_t)tp * sstride + j] = v;
                prow[j] = v;
                if (j == k + 1) fn[tp] = v;
            }
            if (threadIdx.x == 0) used[tp] = 1;
        }
        cl.sync();
        if (c != owner) {
            const S* rp = cl.map_shared_rank(prow, owner);
            for (int j = threadIdx.x; j < s; j += blockDim.x) prow[j] = rp[j];
        }
        __syncthreads();
        const S d = prow[k];
        for (int tl = tl0, j = j0; tl < rows_loc;) {
            if (!(c == owner && tl == tp)) {
                const S f = fc[tl];
                if (j == k) slab[(size_t)tl * sstride + k] = sc_neg(sc_mul(f, d));
                else {
                    const S v = sc_fms(slab[(size_t)tl * sstride + j], f, prow[j]);
                    slab[(size_t)tl * sstride + j] = v;
                    if (j == k + 1) fn[tl] = v;
                }
            }
            tl += dr;
            j += dc;
            if (j >= s) { j -= s; ++tl; }
        }
        __syncthreads();
    }
    // write Pi = S A^{-1} S: A^{-1}[k][p_j] = R[p_k][j]; local row i = p_k for k = pinv(i), found
    // once per row (into `used`, free after the elimination)
    T* Pi = L.Pi + L.pioff[e];
    const int ld = L.pild[e];
    alpha = s_alpha;
    for (int tl = threadIdx.x; tl < rows_loc; tl += blockDim.x) {
        const int i = c + tl * C;
        int kk = 0;
        while (kk < s - 1 && perm[kk] != i) ++kk;
        used[tl] = kk;
    }
    __syncthreads();
    for (int tl = tl0, j = j0; tl < rows_loc;) {
        const int kk = used[tl];
        const int col = perm[j];
        const double sc = (kk >= n ? alpha : 1.0) * (col >= n ? alpha : 1.0);
        Pi[(size_t)kk * ld + col] = (T)(sc * (double)slab[(size_t)tl * sstride + j]);
        tl += dr;
        j += dc;
        if (j >= s) { j -= s; ++tl; }
    }
    if (threadIdx.x == 0 && c == 0) {
        atomicAdd(&L.counters[2], 2.0 * s * (double)s * s);
        atomicAdd(&L.counters[3], 2.0 * s * (double)s * s);
    }
    cl.sync();  // no block leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------------------------
// k_panel: X = Pi_e[:, 0:n] B_q for each neighbour q, X_y = -Pi_e[:, n:s]; panels for the solve
// ---------------------------------------------------------------------------------------------
// CTA GEMM of the panel, Schur and compression steps: in the working precision (DF = false), or,
// for FP64 level data with gemm_dfl set (DF = true), in double-float on the FP32 pipe (operands
// split while they are staged, FP64 epilogue). DF is a template parameter so that each kernel
// instantiation carries one GEMM only (registers, hence occupancy).
template <typename T, bool DF, class LA, class LB, class EPI>
IFMM_DEVINL void factor_gemm(const LevelView<T>& L, int M, int N, int K, LA la, LB lb, EPI epi, void* sm, int tile0,
                             int tstride) {
    using Acc = typename AccOf<T>::type;
    (void)L;
    if constexpr (DF && std::is_same<T, double>::value) {
        cta_gemm<dfl>(M, N, K, la, lb, [&](int i, int j, dfl v) { epi(i, j, (double)v); }, (dfl*)sm, tile0, tstride);
    } else {
        cta_gemm<Acc>(M, N, K, la, lb, epi, (Acc*)sm, tile0, tstride);
    }
}

template <typename T, bool DF>
__global__ void __launch_bounds__(kThreads) k_panel(LevelView<T> L0, BoxList<T> bl, int colour) {
    const LevelView<T>& L = bl.view(L0, blockIdx.x);
    using Acc = typename AccOf<T>::type;
    using GS = std::conditional_t<DF && std::is_same<T, double>::value, dfl, Acc>;
    __shared__ GS sm[gemm_smem<GS>::value];
    const int e = bl.box(blockIdx.x);
    const int d = blockIdx.y;
    const Cell ce = cell_of(e, L.side, L.dim);
    const Cell cq = cell_dir(ce, d, L.dim);
    if (!cell_in(cq, L.side)) return;
    const int n = L.n[e], r = L.r[e], s = n + r;
    T* X = L.Xs + L.xsoff[e];
    const int ldx = L.xsld[e];
    const T* Pi = L.Pi + L.pioff[e];
    const int ldpi = L.pild[e];
    if (d == L.ctr) {
        if (blockIdx.z != 0) return;
        int cy = xcol_offset(L, ce, L.ctr);
        for (int t = threadIdx.x; t < s * r; t += blockDim.x) {
            int i = t / r, j = t - i * r;
            X[(size_t)i * ldx + cy + j] = -Pi[(size_t)i * ldpi + n + j];
        }
        return;
    }
    const int q = cell_index(cq, L.side);
    const int wq = active_width(L, q, colour);
    int ldb;
    const T* B = block_at(L, e, q, ldb);
    if (blockIdx.z == 0) {
        // B panel (row P2P_e at q's active unknown), n x wq, kept for the back substitution
        T* Bp = L.Bp + L.bpoff[(int64_t)e * L.nd + d];
        for (int t = threadIdx.x; t < n * wq; t += blockDim.x) {
            int i = t / wq, j = t - i * wq;
            Bp[t] = B[(size_t)i * ldb + j];
        }
        // C panel (q's active equation at x_e), wq x n, kept for the forward replay and the Schur step
        int ldc;
        const T* C = block_at(L, q, e, ldc);
        T* Cp = L.Cp + L.cpoff[(int64_t)e * L.nd + d];
        for (int t = threadIdx.x; t < wq * n; t += blockDim.x) {
            int i = t / n, j = t - i * n;
            Cp[t] = C[(size_t)i * ldc + j];
        }
    }
    const int cx = xcol_offset(L, ce, d);
    factor_gemm<T, DF>(
        L, s, wq, n, [&](int i, int k) { return Pi[(size_t)i * ldpi + k]; },
        [&](int k, int j) { return B[(size_t)k * ldb + j]; },
        [&](int i, int j, Acc v) { X[(size_t)i * ldx + cx + j] = (T)v; }, sm, blockIdx.z, gridDim.z);
    if (threadIdx.x == 0 && blockIdx.z == 0) {
        atomicAdd(&L.counters[2], 2.0 * s * (double)wq * n);
        atomicAdd(&L.counters[4], 2.0 * s * (double)wq * n);
    }
}

// ---------------------------------------------------------------------------------------------
// k_schur: one (p, q) pair of neighbours of e per block (p, q in N_e; dp == ctr is row M2L_e)
// ---------------------------------------------------------------------------------------------
// GM selects the product: 0 = the working precision (FP64 exact extent, or FP32), 1 = double-float
// on the FP32 pipe, 2 = the tensor cores (ifmm_tc.cuh: digit-split bf16 MMAs, 128 threads, dynamic
// shared memory and tensor memory taken only by the blocks that multiply)
template <typename T, int GM>
__global__ void __launch_bounds__(GM == 2 ? tc::kThreads : kThreads) k_schur(LevelView<T> L0, BoxList<T> bl, int colour) {
    const LevelView<T>& L = bl.view(L0, blockIdx.x);
    using Acc = typename AccOf<T>::type;
    using GS = std::conditional_t<GM == 1 && std::is_same<T, double>::value, dfl, Acc>;
    __shared__ GS sm[GM == 2 ? 1 : gemm_smem<GS>::value];
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    auto gemm = [&](int M, int N, int K, auto la, auto lb, auto epi) {
        if constexpr (GM == 2) {
            tc::Ctx c;
            tc::ctx_init(c, tc_smem, L.status);
            tc::tc_gemm(c, M, N, K, la, lb, epi, blockIdx.z, gridDim.z);
            tc::ctx_release(c);
        } else {
            factor_gemm<T, GM == 1>(L, M, N, K, la, lb, epi, sm, blockIdx.z, gridDim.z);
        }
    };
    const int e = bl.box(blockIdx.x);
    const int dp = blockIdx.y / L.nd, dq = blockIdx.y % L.nd;
    const Cell ce = cell_of(e, L.side, L.dim);
    const Cell cp = cell_dir(ce, dp, L.dim), cq = cell_dir(ce, dq, L.dim);
    if (!cell_in(cp, L.side) || !cell_in(cq, L.side)) return;
    const int p = cell_index(cp, L.side), q = cell_index(cq, L.side);
    const int n = L.n[e], r = L.r[e];
    const T* X = L.Xs + L.xsoff[e];
    const int ldx = L.xsld[e];
    if (dp == L.ctr) {
        // row M2L_e has -I at z_e: A[M2L_e, gamma] = X_gamma[z rows]
        if (blockIdx.z != 0) return;
        int ld;
        T* dst = block_at(L, e, q, ld);
        const int w = (dq == L.ctr) ? r : active_width(L, q, colour);
        const int cx = xcol_offset(L, ce, dq);
        for (int t = threadIdx.x; t < r * w; t += blockDim.x) {
            int i = t / w, j = t - i * w;
            dst[(size_t)i * ld + j] = X[(size_t)(n + i) * ldx + cx + j];
        }
        return;
    }
    // symmetric kernel: the (q, p) block is the transpose of the (p, q) block, written by that block
    if (L.symmetric && dq != L.ctr && dp > dq) return;
    const int wp = active_width(L, p, colour);
    const T* C = L.Cp + L.cpoff[(int64_t)e * L.nd + dp];
    const int cx = xcol_offset(L, ce, dq);
    if (dq == L.ctr) {
        // new column y_e in row rho_p: M2P_pe or M2L_pe = -C_p X_y[x rows]
        int ld;
        T* dst = block_at(L, p, e, ld);
        gemm(wp, r, n, [&](int i, int k) { return C[(size_t)i * n + k]; },
             [&](int k, int j) { return X[(size_t)k * ldx + cx + j]; },
             [&](int i, int j, Acc v) { dst[(size_t)i * ld + j] = (T)(-v); });
        if (threadIdx.x == 0 && blockIdx.z == 0) {
            atomicAdd(&L.counters[0], 2.0 * wp * (double)r * n);
            atomicAdd(&L.counters[1], (double)sizeof(T) * ((double)wp * n + (double)n * r + (double)wp * r));
            atomicAdd(&L.counters[2], 2.0 * wp * (double)r * n);
        }
        return;
    }
    const int wq = active_width(L, q, colour);
    const int dist = cheb_dist(cp, cq);
    const bool Ep = cell_colour(cp) < colour, Eq = cell_colour(cq) < colour;
    if (dist <= 1 || (Ep && Eq)) {
        // neighbours: dense update in place; both eliminated: M2L_pq updated directly
        int ld, ld2 = 0;
        T* dst = block_at(L, p, q, ld);
        T* dst2 = (L.symmetric && p != q) ? block_at(L, q, p, ld2) : nullptr;
        gemm(wp, wq, n, [&](int i, int k) { return C[(size_t)i * n + k]; },
             [&](int k, int j) { return X[(size_t)k * ldx + cx + j]; },
             [&](int i, int j, Acc v) {
                 dst[(size_t)i * ld + j] = (T)((Acc)dst[(size_t)i * ld + j] - v);
                 if (dst2) dst2[(size_t)j * ld2 + i] = (T)((Acc)dst2[(size_t)j * ld2 + i] - v);
             });
    } else {
        T* F = L.Fs + fill_off(L, e, dp, dq);
        gemm(wp, wq, n, [&](int i, int k) { return C[(size_t)i * n + k]; },
             [&](int k, int j) { return X[(size_t)k * ldx + cx + j]; },
             [&](int i, int j, Acc v) { F[(size_t)i * wq + j] = (T)(-v); });
    }
    if (threadIdx.x == 0 && blockIdx.z == 0) {
        double fl = 2.0 * wp * (double)wq * n;
        atomicAdd(&L.counters[0], fl);
        const double mirror = (L.symmetric && p != q && (dist <= 1 || (Ep && Eq))) ? 2.0 : 1.0;
        atomicAdd(&L.counters[1], (double)sizeof(T) * ((double)wp * n + (double)n * wq + 2.0 * mirror * wp * wq));
        atomicAdd(&L.counters[2], fl);
    }
}

// ---------------------------------------------------------------------------------------------
// k_compress: extend W_q for the well-separated fill of uneliminated neighbour q of e
// ---------------------------------------------------------------------------------------------
// element operations of the compression's Gram-Schmidt, in FP64 (or FP32) or double-float
IFMM_DEVINL void gs_fma(double& s, double a, double b) { s = fma(a, b, s); }
IFMM_DEVINL void gs_fma(float& s, float a, float b) { s = fmaf(a, b, s); }
IFMM_DEVINL void gs_fma(dfl& s, dfl a, dfl b) { dfl_fma_acc(s, a, b); s = dfl_norm(s); }
IFMM_DEVINL double gs_shfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
IFMM_DEVINL float gs_shfl(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
IFMM_DEVINL dfl gs_shfl(dfl v, int o) {
    return dfl(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
IFMM_DEVINL double gs_d(double v) { return v; }
IFMM_DEVINL double gs_d(float v) { return (double)v; }
IFMM_DEVINL double gs_d(dfl v) { return (double)v; }
// r - s u
IFMM_DEVINL double gs_axpy(double r, double s, double u) { return fma(-s, u, r); }
IFMM_DEVINL float gs_axpy(float r, float s, float u) { return fmaf(-s, u, r); }
IFMM_DEVINL dfl gs_axpy(dfl r, dfl s, dfl u) {
    dfl_fma_acc(r, dfl(-s.hi, -s.lo), u);
    return dfl_norm(r);
}

// gscr: the FP64 work arrays live in the colour's global scratch (L.Cws) instead of shared memory
// (wide fills, whose arrays exceed the shared-memory budget of the launch)
// C > 1: one compression is spread over a cluster of C blocks (few boxes per colour: the upper
// levels). Block c owns the columns [c mc, (c + 1) mc) of the stacked fill (mc = ceil(m / C)): it
// gathers, projects and updates those columns and keeps their norms; the pivot column is chosen
// over the cluster (candidates exchanged through distributed shared memory, one cluster barrier
// per step) and read from global memory past L1; every block then forms the same direction u
// (same operations in the same order) and writes the same basis column. Per column the arithmetic
// is the single-block one, so the result is the same bit for bit.
constexpr int kMaxPartners = 19;
constexpr int kGB = 4;   // column elements a thread of the Gram-Schmidt loads ahead
IFMM_DEVINL double load_cg(const double* p) { return __ldcg(p); }
IFMM_DEVINL float load_cg(const float* p) { return __ldcg(p); }
IFMM_DEVINL dfl load_cg(const dfl* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return dfl(v.x, v.y);
}
template <typename T, bool DF>
__global__ void __launch_bounds__(kThreads) k_compress(LevelView<T> L0, BoxList<T> bl, int colour, int gscr, int C) {
    namespace cg = cooperative_groups;
    const int crank = C > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const LevelView<T>& L = bl.view(L0, blockIdx.x / C);
    using Acc = typename AccOf<T>::type;
    extern __shared__ double csm_dyn[];  // u (nq), per-warp coefficients (8 * RC), column norms (m)
    using GS = std::conditional_t<DF && std::is_same<T, double>::value, dfl, Acc>;
    __shared__ GS gsm[gemm_smem<GS>::value];
    __shared__ double vred[32];
    __shared__ int ired[32];
    __shared__ double s_cval[2];   // this block's pivot candidate, double-buffered by step parity
    __shared__ int s_cidx[2];
    // the cluster's best (value, index) over the blocks' candidates of parity slot sl: ties to the
    // lowest column (the single-block rule); read by every block after the cluster barrier
    auto cluster_best = [&](int sl, double* val) {
        cg::cluster_group cl = cg::this_cluster();
        return cluster_pick(cl, &s_cval[sl], &s_cidx[sl], C, val);
    };
    const int e = bl.box(blockIdx.x / C);
    const int dq = blockIdx.y;
    if (dq == L.ctr) return;
    const Cell ce = cell_of(e, L.side, L.dim);
    const Cell cq = cell_dir(ce, dq, L.dim);
    if (!cell_in(cq, L.side) || cell_colour(cq) < colour) return;
    const int q = cell_index(cq, L.side);
    // partners: the neighbours of e at Chebyshev distance 2 from q (at most 5 in 2D, 19 in 3D)
    int parts[kMaxPartners], np = 0;
    for (int dp = 0; dp < L.nd; ++dp) {
        if (dp == L.ctr || dp == dq) continue;
        const Cell cp = cell_dir(ce, dp, L.dim);
        if (!cell_in(cp, L.side)) continue;
        if (cheb_dist(cp, cq) == 2) parts[np++] = dp;
    }
    if (np == 0) return;
    const int nq = L.n[q];
    const int rq0 = L.r[q];
    const int RC = L.RC;
    // S_q = [F_qp (nq x wp), F_pq^T (nq x wp)] over the partners p. For a symmetric kernel the Schur
    // update writes each fill pair as a block and its transpose (F_pq^T = F_qp bit for bit), so the
    // row fills F_qp alone make up S_q (reading R2)
    const bool half = L.symmetric != 0;
    int wps[kMaxPartners], m = 0;
    for (int t = 0; t < np; ++t) {
        int dp = parts[t];
        int p = cell_index(cell_dir(ce, dp, L.dim), L.side);
        wps[t] = active_width(L, p, colour);
        m += (half ? 1 : 2) * wps[t];
    }
    if (nq == 0 || m == 0) return;
    // this block's columns [j0, j1) (all of them for a single block)
    const int mc = (m + C - 1) / C;
    const int j0 = min(m, crank * mc), j1 = min(m, j0 + mc), mloc = j1 - j0;
    T* R = L.Rs + L.rsoff[(int64_t)e * L.nd + dq];
    double* csm = gscr ? L.Cws + L.cwsoff[(int64_t)e * L.nd + dq] : csm_dyn;
    {
        int c0 = 0;
        for (int t = 0; t < np; ++t) {
            int dp = parts[t], wp = wps[t];
            if (c0 >= j1 || c0 + (half ? 1 : 2) * wp <= j0) {   // no column of this block
                c0 += (half ? 1 : 2) * wp;
                continue;
            }
            if (half) {
                // F_qp is stored as is (dq < dp, nq x wp) or as its transpose F_pq (wp x nq); either
                // way element u of the stored block is read in order (coalesced), four per thread
                // before their stores so that the loads are in flight together
                const bool direct = dq < dp;
                const T* F = L.Fs + (direct ? fill_off(L, e, dq, dp) : fill_off(L, e, dp, dq));
                const int tot = nq * wp;
                constexpr int kB = 4;
                for (int u0 = threadIdx.x; u0 < tot; u0 += kB * (int)blockDim.x) {
                    T v[kB];
                    int64_t dst[kB];
#pragma unroll
                    for (int k = 0; k < kB; ++k) {
                        const int u = u0 + k * (int)blockDim.x;
                        dst[k] = -1;
                        if (u < tot) {
                            const int a = direct ? u / wp : u / nq, b = direct ? u - a * wp : u - a * nq;
                            const int i = direct ? a : b, j = direct ? b : a;
                            v[k] = F[u];
                            if (c0 + j >= j0 && c0 + j < j1) dst[k] = (int64_t)i * m + c0 + j;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kB; ++k)
                        if (dst[k] >= 0) R[dst[k]] = v[k];
                }
            } else {
                for (int u = threadIdx.x; u < nq * wp; u += blockDim.x) {
                    int i = u / wp, j = u - i * wp;
                    if (c0 + j >= j0 && c0 + j < j1)
                        R[(size_t)i * m + c0 + j] = fill_at(L, e, dq, dp, nq, wp, i, j);            // F_qp
                    if (c0 + wp + j >= j0 && c0 + wp + j < j1)
                        R[(size_t)i * m + c0 + wp + j] = fill_at(L, e, dp, dq, wp, nq, j, i);       // F_pq^T
                }
            }
            c0 += (half ? 1 : 2) * wp;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // reference norm: largest column norm of S_q, one column per thread (consecutive threads read
    // consecutive columns of a row: coalesced; a warp per column reads 32 rows m apart)
    double nmx = 0.0;
    for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) {
        double s = 0.0;
#pragma unroll 4
        for (int i = 0; i < nq; ++i) { const double v = (double)R[(size_t)i * m + j]; s = fma(v, v, s); }
        nmx = fmax(nmx, sqrt(s));
    }
    double smax = block_max(nmx, vred);
    if (C > 1) {
        // the largest over the cluster (slot 0 holds it, read by every block before the second
        // barrier, after which slot 0 may be reused)
        if (threadIdx.x == 0) { s_cval[0] = smax; s_cidx[0] = 0; }
        cg::this_cluster().sync();
        double v;
        (void)cluster_best(0, &v);
        smax = v;
        cg::this_cluster().sync();
    }
    if (!(smax > 0.0)) return;
    const double tau = L.eps * (L.tau_ref == 1 ? L.sA : smax);
    T* W = L.W + L.voff[q] * RC;
    double* coef = csm + nq;  // 8 warps x RC
    // R <- (I - W W^T) R: once in FP64 (the basis is orthonormal to working precision), twice in
    // FP32. With the column fills alone (half) the second half of R's scratch is free and holds
    // C = W^T R, and the projection is two CTA GEMMs (in double-float for gemm_dfl); otherwise
    // classical Gram-Schmidt per column.
    const int passes = sizeof(T) == 8 ? 1 : 2;
    if (half && passes == 1 && rq0 > 0) {
        // (this block's columns: column j of the products is column j0 + j of R)
        T* Cm = R + (size_t)nq * m + j0;
        T* Rj = R + j0;
        factor_gemm<T, DF>(
            L, rq0, mloc, nq, [&](int i, int k) { return W[(size_t)k * RC + i]; },
            [&](int k, int j) { return Rj[(size_t)k * m + j]; },
            [&](int i, int j, Acc v) { Cm[(size_t)i * m + j] = (T)v; }, gsm, 0, 1);
        __syncthreads();
        factor_gemm<T, DF>(
            L, nq, mloc, rq0, [&](int i, int k) { return W[(size_t)i * RC + k]; },
            [&](int k, int j) { return Cm[(size_t)k * m + j]; },
            [&](int i, int j, Acc v) { Rj[(size_t)i * m + j] = (T)((Acc)Rj[(size_t)i * m + j] - v); }, gsm, 0, 1);
        __syncthreads();
    }
    for (int pass = 0; pass < passes && rq0 > 0 && !(half && passes == 1); ++pass) {
        for (int j = j0 + warp; j < j1; j += nw) {
            double* c = coef + warp * RC;
            for (int t = 0; t < rq0; ++t) {
                Acc s = 0;
                for (int i = lane; i < nq; i += 32) s += (Acc)W[(size_t)i * RC + t] * (Acc)R[(size_t)i * m + j];
                s = warp_sum(s);
                if (lane == 0) c[t] = (double)s;
            }
            __syncwarp();
            for (int i = lane; i < nq; i += 32) {
                Acc acc = (Acc)R[(size_t)i * m + j];
                for (int t = 0; t < rq0; ++t) acc -= (Acc)W[(size_t)i * RC + t] * (Acc)c[t];
                R[(size_t)i * m + j] = (T)acc;
            }
            __syncwarp();
        }
        __syncthreads();
    }
    const int limit = min(nq, RC);
    double* u = csm;
    double* nrm2 = coef + 8 * RC;   // squared norms of this block's columns of R (column j0 + j at j)
    // the column work of the Gram-Schmidt: FP64, or double-float on the FP32 pipe when the products
    // are double-float (the basis, the re-orthogonalisation, the norms that decide the pivots and the
    // ranks, and the threshold test stay FP64)
    using E = std::conditional_t<DF && std::is_same<T, double>::value, dfl, Acc>;
    E* Re = reinterpret_cast<E*>(R);
    E* ue = reinterpret_cast<E*>(nrm2 + (C > 1 ? mloc : m));   // u in E (nq entries)
    if constexpr (std::is_same<E, dfl>::value) {
        // R to double-float in place (the split works on the bit pattern: no FP64 arithmetic); a
        // single block converts whole rows without an index division per element
        if (mloc == m) {
            for (int t = threadIdx.x; t < nq * m; t += blockDim.x) Re[t] = dfl((double)R[t]);
        } else {
            for (int t = threadIdx.x; t < nq * mloc; t += blockDim.x) {
                const int i = t / mloc, j = j0 + (t - i * mloc);
                Re[(size_t)i * m + j] = dfl((double)R[(size_t)i * m + j]);
            }
        }
        __syncthreads();
    }
    // g threads per column (a power of two dividing 32; more when the columns are few; set by the
    // whole width m so that a column is summed in the same order in a cluster), ngr groups; every
    // warp runs the same number of column rounds so the group shuffles converge
    int g = 1;
    while (g < 8 && g * 2 * m <= (int)blockDim.x) g *= 2;
    const int ngr = (int)blockDim.x / g, gid = (int)threadIdx.x / g, gl = (int)threadIdx.x % g;
    const int rounds = (mloc + ngr - 1) / ngr;
    auto group_sum = [&](E v) {
        for (int o = g >> 1; o > 0; o >>= 1) v = v + gs_shfl(v, o);
        return v;
    };
    for (int rd = 0; rd < rounds; ++rd) {
        const int j = j0 + gid + rd * ngr;
        E sq = E(0);
        if (j < j1) {
            int i = gl;
            for (; i + (kGB - 1) * g < nq; i += kGB * g) {
                E x[kGB];
#pragma unroll
                for (int k = 0; k < kGB; ++k) x[k] = Re[(size_t)(i + k * g) * m + j];
#pragma unroll
                for (int k = 0; k < kGB; ++k) gs_fma(sq, x[k], x[k]);
            }
            for (; i < nq; i += g) { const E v = Re[(size_t)i * m + j]; gs_fma(sq, v, v); }
        }
        sq = group_sum(sq);
        if (j < j1 && gl == 0) nrm2[j - j0] = gs_d(sq);
    }
    __syncthreads();
    int add = 0;
    for (int step = 0;; ++step) {
        // largest remaining column norm, ties to the lowest column (reading R2). The norms are
        // recomputed from the updated columns at every step, so the pivot is chosen on exact norms
        // as in the oracle: an estimate (a downdated norm) lets nearly equal columns swap order,
        // and a different pivot order leaves a different remainder below the threshold.
        double best = -1.0;
        int bi = -1;
        for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) {
            const double v = nrm2[j - j0];
            if (bi < 0 || v > best) { best = v; bi = j; }
        }
        double b2;
        int jb = block_argmax(best, bi, vred, ired, &b2);
        if (C > 1) {
            if (threadIdx.x == 0) { s_cval[step & 1] = b2; s_cidx[step & 1] = jb; }
            // also orders this block's column updates (global memory) before the others' reads
            cg::this_cluster().sync();
            jb = cluster_best(step & 1, &b2);
        }
        if (jb < 0) break;
        const double bv = sqrt(b2);
        if (!(bv > tau)) break;
        if (rq0 + add >= limit) {
            if (limit < nq && threadIdx.x == 0 && crank == 0) atomicOr(L.status, DEV_ERR_OVERFLOW);
            break;
        }
        const int rc = rq0 + add;
        const double ib = 1.0 / bv;
        // (the pivot column may belong to another block of the cluster: read past L1)
        for (int i = threadIdx.x; i < nq; i += blockDim.x) u[i] = gs_d(load_cg(Re + (size_t)i * m + jb)) * ib;
        __syncthreads();
        // re-orthogonalise u against the current basis, twice (one thread per basis vector for the
        // coefficients, one per row for the update)
        for (int pass = 0; pass < 2; ++pass) {
            for (int t = threadIdx.x; t < rc; t += blockDim.x) {
                double sc = 0.0;
#pragma unroll 4
                for (int i = 0; i < nq; ++i) sc += (double)W[(size_t)i * RC + t] * u[i];
                coef[t] = sc;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nq; i += blockDim.x) {
                double acc = u[i];
#pragma unroll 4
                for (int t = 0; t < rc; ++t) acc -= (double)W[(size_t)i * RC + t] * coef[t];
                u[i] = acc;
            }
            __syncthreads();
        }
        double nn = 0.0;
        for (int i = threadIdx.x; i < nq; i += blockDim.x) nn += u[i] * u[i];
        nn = block_sum(nn, vred);
        const double nu = sqrt(nn);
        if (!(nu >= 0.5)) {
            // numerically inside the current span: drop this column (its owner clears it)
            if (jb >= j0 && jb < j1) {
                for (int i = threadIdx.x; i < nq; i += blockDim.x) Re[(size_t)i * m + jb] = E(0);
                if (threadIdx.x == 0) nrm2[jb - j0] = 0.0;
            }
            __syncthreads();
            continue;
        }
        const double inu = 1.0 / nu;
        // every block of a cluster writes the same basis column (the same values), so each reads
        // back its own writes in the next re-orthogonalisation
        for (int i = threadIdx.x; i < nq; i += blockDim.x) {
            u[i] *= inu;
            W[(size_t)i * RC + rc] = (T)u[i];
            ue[i] = E(u[i]);
        }
        __syncthreads();
        // remove u from every column; the squared norm of the updated column is summed in the same
        // pass (one more multiply-add per element, no extra memory traffic)
        for (int rd = 0; rd < rounds; ++rd) {
            const int j = j0 + gid + rd * ngr;
            // kGB elements of the column loaded together before they are used (stores to R would
            // otherwise keep the compiler from hoisting the next loads); same order of operations
            E sp = E(0);
            if (j < j1) {
                int i = gl;
                for (; i + (kGB - 1) * g < nq; i += kGB * g) {
                    E x[kGB];
#pragma unroll
                    for (int k = 0; k < kGB; ++k) x[k] = Re[(size_t)(i + k * g) * m + j];
#pragma unroll
                    for (int k = 0; k < kGB; ++k) gs_fma(sp, ue[i + k * g], x[k]);
                }
                for (; i < nq; i += g) gs_fma(sp, ue[i], Re[(size_t)i * m + j]);
            }
            sp = group_sum(sp);
            E sq = E(0);
            if (j < j1) {
                int i = gl;
                for (; i + (kGB - 1) * g < nq; i += kGB * g) {
                    E x[kGB];
#pragma unroll
                    for (int k = 0; k < kGB; ++k) x[k] = Re[(size_t)(i + k * g) * m + j];
#pragma unroll
                    for (int k = 0; k < kGB; ++k) {
                        const E v = gs_axpy(x[k], sp, ue[i + k * g]);   // R_ij - sp u_i
                        Re[(size_t)(i + k * g) * m + j] = v;
                        gs_fma(sq, v, v);
                    }
                }
                for (; i < nq; i += g) {
                    const E v = gs_axpy(Re[(size_t)i * m + j], sp, ue[i]);
                    Re[(size_t)i * m + j] = v;
                    gs_fma(sq, v, v);
                }
            }
            sq = group_sum(sq);
            if (j < j1 && gl == 0) nrm2[j - j0] = gs_d(sq);
        }
        __syncthreads();
        ++add;
    }
    if (threadIdx.x == 0 && crank == 0) {
        L.r[q] = rq0 + add;
        // projection onto the complement of the old basis (two products of nq x m x rq0 per pass)
        // and the pivoted Gram-Schmidt: per appended direction a dot product, an update and a norm
        // of every column (6 nq m) plus two re-orthogonalisations against the basis (8 nq rc),
        // and the last, unsuccessful search (6 nq m)
        const double proj = 4.0 * passes * (double)nq * m * rq0;
        const double gs = 6.0 * (double)nq * m * (add + 1) + 8.0 * (double)nq * ((double)add * rq0 + 0.5 * add * (add - 1));
        atomicAdd(&L.counters[2], proj + gs);
        atomicAdd(&L.counters[5], proj + gs);
        atomicAdd(&L.counters[7], proj);
        atomicAdd(&L.counters[8], 8.0 * (double)nq * ((double)add * rq0 + 0.5 * add * (add - 1)));
    }
    // no block leaves while another may still read its candidate slots
    if (C > 1) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------------------------
// k_redirect: M2L_pq += (W_p^T) F (W_q) for a well-separated pair with fill
// ---------------------------------------------------------------------------------------------
template <typename T, bool DF>
__global__ void __launch_bounds__(kThreads) k_redirect(LevelView<T> L0, BoxList<T> bl, int colour) {
    const LevelView<T>& L = bl.view(L0, blockIdx.x);
    using Acc = typename AccOf<T>::type;
    using GS = std::conditional_t<DF && std::is_same<T, double>::value, dfl, Acc>;
    __shared__ GS sm[gemm_smem<GS>::value];
    const int e = bl.box(blockIdx.x);
    const int dp = blockIdx.y / L.nd, dq = blockIdx.y % L.nd;
    if (dp == L.ctr || dq == L.ctr || dp == dq) return;
    const Cell ce = cell_of(e, L.side, L.dim);
    const Cell cp = cell_dir(ce, dp, L.dim), cq = cell_dir(ce, dq, L.dim);
    if (!cell_in(cp, L.side) || !cell_in(cq, L.side)) return;
    if (cheb_dist(cp, cq) != 2) return;
    const bool Ep = cell_colour(cp) < colour, Eq = cell_colour(cq) < colour;
    if (Ep && Eq) return;
    if (L.symmetric && dp > dq) return;   // M2L_qp += G_pq^T below
    const int p = cell_index(cp, L.side), q = cell_index(cq, L.side);
    const int wp = Ep ? L.r[p] : L.n[p];
    const int wq = Eq ? L.r[q] : L.n[q];
    const int rp = L.r[p], rq = L.r[q];
    const int RC = L.RC;
    const int64_t fo = fill_off(L, e, dp, dq);
    const T* F = L.Fs + fo;   // wp x wq
    T* F2 = L.Fs2 + fo;       // wp x rq
    int ld, ld2 = 0;
    T* M = block_at(L, p, q, ld);
    T* M2 = L.symmetric ? block_at(L, q, p, ld2) : nullptr;
    const T* Wq = L.W + L.voff[q] * RC;
    const T* Wp = L.W + L.voff[p] * RC;
    const T* T1 = F;
    int ld1 = wq;
    if (!Eq) {
        factor_gemm<T, DF>(
            L, wp, rq, wq, [&](int i, int k) { return F[(size_t)i * wq + k]; },
            [&](int k, int j) { return Wq[(size_t)k * RC + j]; },
            [&](int i, int j, Acc v) { F2[(size_t)i * rq + j] = (T)v; }, sm, 0, 1);
        __syncthreads();
        T1 = F2;
        ld1 = rq;
    }
    if (!Ep) {
        factor_gemm<T, DF>(
            L, rp, rq, wp, [&](int i, int k) { return Wp[(size_t)k * RC + i]; },
            [&](int k, int j) { return T1[(size_t)k * ld1 + j]; },
            [&](int i, int j, Acc v) {
                M[(size_t)i * ld + j] = (T)((Acc)M[(size_t)i * ld + j] + v);
                if (M2) M2[(size_t)j * ld2 + i] = (T)((Acc)M2[(size_t)j * ld2 + i] + v);
            },
            sm, 0, 1);
    } else {
        for (int t = threadIdx.x; t < rp * rq; t += blockDim.x) {
            int i = t / rq, j = t - i * rq;
            Acc v = (Acc)T1[(size_t)i * ld1 + j];
            M[(size_t)i * ld + j] = (T)((Acc)M[(size_t)i * ld + j] + v);
            if (M2) M2[(size_t)j * ld2 + i] = (T)((Acc)M2[(size_t)j * ld2 + i] + v);
        }
    }
    if (threadIdx.x == 0) {
        double fl = 2.0 * wp * (double)rq * wq * (Eq ? 0 : 1) + 2.0 * rp * (double)rq * wp * (Ep ? 0 : 1);
        atomicAdd(&L.counters[2], fl);
        atomicAdd(&L.counters[6], fl);
    }
}

// Largest dynamic shared memory a launch of `fn` may use: the device's opt-in limit per block less
// the kernel's static shared memory (queried once per kernel and device).
int dynamic_smem_limit(const void* fn) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> lim;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = lim.find({fn, dev});
    if (it != lim.end()) return it->second;
    int optin = 0;
    cudaFuncAttributes fa{};
    int v = 48 * 1024;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
        v = optin - (int)fa.sharedSizeBytes;
    cudaGetLastError();
    lim[{fn, dev}] = v;
    return v;
}

// Launch of kfn over clusters of c blocks along x (grid.x a multiple of c). Whether the shape can be
// scheduled is asked once per (kernel, c, shared memory); c = 16 (beyond the portable 8) is opted
// into per kernel. False: nothing was launched (the caller takes a smaller cluster or none).
template <typename... KArgs, typename... Args>
bool launch_clustered(void (*kfn)(KArgs...), int c, dim3 grid, size_t smem, cudaStream_t st, Args... args) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t>, int> occ;
    if (c > 8) {
        std::lock_guard<std::mutex> lk(mu);
        const auto key = std::make_tuple((const void*)kfn, -1, (size_t)0);
        if (occ.find(key) == occ.end()) {
            occ[key] = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
            cudaGetLastError();
        }
        if (!occ[key]) return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int active = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        const auto key = std::make_tuple((const void*)kfn, c, smem);
        auto it = occ.find(key);
        if (it != occ.end()) active = it->second;
        else {
            if (cudaOccupancyMaxActiveClusters(&active, kfn, &cfg) != cudaSuccess) active = 0;
            cudaGetLastError();
            occ[key] = active;
        }
    }
    if (active < 1) return false;
    if (cudaLaunchKernelEx(&cfg, kfn, args...) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

__global__ void k_set_flag(int* status, int flag) { atomicOr(status, flag); }

// ---------------------------------------------------------------------------------------------
// Autotuner of the split of the panel and Schur launches: how many blocks share one box's (panel)
// or one pair's (Schur) product, i.e. the output tiles each block takes. A table maps a bucket --
// (kernel, double-float products or not, ceil(log2 nmax), ceil(log2 boxes of the launch)), the
// launch's block size s and its box count -- to the split that ran fastest when it was measured; a
// bucket without an entry takes the fixed rule. A split only changes which block computes which
// output tile, never the arithmetic of a tile, so every split gives the same results bit for bit.
// The table is process-wide (one mutex); tuning records the launches' device times with events.
// ---------------------------------------------------------------------------------------------
namespace tune {
using Key = std::tuple<int, int, int, int>;
std::mutex mu;
std::map<Key, int> table;
int force[2] = {0, 0};   // while tuning: the candidate split of the panel / Schur launches (0: none)
bool recording = false;
struct Rec { Key key; cudaEvent_t e0, e1; };
std::vector<Rec> recs;

int ceil_log2(int v) {
    int b = 0;
    while (b < 30 && (1 << b) < v) ++b;
    return b;
}
// the split of a launch: the forced candidate while tuning, else the table's entry, else the rule
int split(const Key& k, int rule) {
    std::lock_guard<std::mutex> lk(mu);
    const int f = force[std::get<0>(k)];
    if (f > 0) return f;
    auto it = table.find(k);
    return it != table.end() ? it->second : rule;
}
}  // namespace tune

void tune_set_force(int panel, int schur) {
    std::lock_guard<std::mutex> lk(tune::mu);
    tune::force[0] = panel;
    tune::force[1] = schur;
}
void tune_record(bool on) {
    std::lock_guard<std::mutex> lk(tune::mu);
    tune::recording = on;
}
// device milliseconds of the recorded launches, summed per bucket, for one kernel; clears the records
std::map<std::tuple<int, int, int, int>, double> tune_collect(int kernel) {
    std::lock_guard<std::mutex> lk(tune::mu);
    std::map<tune::Key, double> out;
    for (auto& r : tune::recs) {
        float ms = 0.f;
        if (std::get<0>(r.key) == kernel && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) out[r.key] += ms;
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    tune::recs.clear();
    cudaGetLastError();
    return out;
}
void tune_table_set(const std::map<std::tuple<int, int, int, int>, int>& t) {
    std::lock_guard<std::mutex> lk(tune::mu);
    tune::table = t;
}
std::map<std::tuple<int, int, int, int>, int> tune_table_get() {
    std::lock_guard<std::mutex> lk(tune::mu);
    return tune::table;
}

// largest pivot size s = n + r over the boxes of a colour at the time of their elimination (the
// ranks grow on the device), into *out
template <typename T>
__global__ void k_colour_smax(LevelView<T> L, const int* boxes, int nboxes, int* out) {
    __shared__ double vred[32];
    double m = 0.0;
    for (int b = threadIdx.x; b < nboxes; b += blockDim.x) m = fmax(m, (double)(L.n[boxes[b]] + L.r[boxes[b]]));
    m = block_max(m, vred);
    if (threadIdx.x == 0) *out = (int)m;
}

template <typename T>
void launch_factor_colour(const LevelView<T>& L, const int* boxes, int nboxes, int colour, int smax_bound,
                          int exact_sizing, cudaStream_t st, cudaEvent_t* ev, const int2* items,
                          const LevelView<T>* views) {
    if (nboxes <= 0) return;
    // the blocks' boxes: one level of one system, or the items of a batch of systems (then L carries
    // the launch sizes: the largest smax, nmax and RC over the batch)
    const BoxList<T> bl{boxes, items, views};
    // size the pivot launch by the colour's actual largest pivot (the level bound nmax + min(nmax,
    // RC) is reached only when a basis fills up); status[2] is the scratch word
    int smax = smax_bound;
    // (the readback waits for the stream: with exact_sizing = 0, as when many systems share the GPU
    // and the pause would idle this system's stream, the level bound is used)
    if (exact_sizing && smax_bound >= 96) {
        k_colour_smax<T><<<1, 256, 0, st>>>(L, boxes, nboxes, L.status + 2);
        count_launches(1);
        int hs = 0;
        if (cudaMemcpyAsync(&hs, L.status + 2, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess && hs > 0 && hs <= smax_bound)
            smax = hs;
    }
    size_t base = (size_t)smax * sizeof(double) + (size_t)((smax + 1) / 2) * sizeof(double);
    size_t full = base + (size_t)smax * smax * sizeof(double);
    int use_smem = full <= 200 * 1024 ? 1 : 0;
    size_t smem = use_smem ? full : base;
    static std::atomic<bool> attr_set[2] = {false, false};
    if (!attr_set[sizeof(T) == 8].load()) {
        cudaFuncSetAttribute(k_pivot<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096);
        // set once to the largest size any launch may use: host threads factoring different systems
        // launch concurrently, so a per-launch setting could be lowered under another's launch
        cudaFuncSetAttribute(k_compress<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dynamic_smem_limit((const void*)k_compress<T, false>));
        cudaFuncSetAttribute(k_compress<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dynamic_smem_limit((const void*)k_compress<T, true>));
        cudaGetLastError();
        attr_set[sizeof(T) == 8].store(true);
    }
    // large pivot blocks and few boxes: one cluster of C blocks per box
    int C = 1, slab_global = 0;
    auto cl_bytes = [&](int cc, int glob) {
        const size_t rows = (size_t)(smax + cc - 1) / cc;
        return (glob ? 0 : rows * smax * sizeof(double)) + (smax + 2 * rows) * sizeof(double) + (smax + rows) * sizeof(int);
    };
    if (smax >= 96) {
        // few boxes: spread each over several SMs (up to 16 at the upper levels); many boxes: keep
        // a CTA within 72 KB so that three share an SM (a pivot is a chain of s dependent steps;
        // resident CTAs hide it)
        while (C < 8 && nboxes * C < 2 * num_sms()) C *= 2;
        if (C == 8 && nboxes * 8 < num_sms()) C = 16;
        while (C < 8 && cl_bytes(C, 0) > 72 * 1024) C *= 2;
    }
    if (ev) cudaEventRecord(ev[0], st);
    if (C > 1) {
        static std::atomic<bool> cl_attr[2] = {false, false};
        if (!cl_attr[sizeof(T) == 8].load()) {
            cudaFuncSetAttribute(k_pivot_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096);
            cl_attr[sizeof(T) == 8].store(true);
        }
    }
    // a cluster shape that cannot be scheduled, or a refused launch, falls back to 8 blocks, then to
    // one block per box
    for (bool done = false; C > 1 && !done;) {
        slab_global = cl_bytes(C, 0) > 200 * 1024 ? 1 : 0;   // slab rows in the FP64 workspace (L2)
        if (!(slab_global && !L.pws))
            done = launch_clustered(k_pivot_cluster<T>, C, dim3((unsigned)(nboxes * C)), cl_bytes(C, slab_global), st,
                                    L, bl, C, smax, slab_global);
        if (!done) C = C > 8 ? 8 : 1;
    }
    if (C == 1) {
        k_pivot<T><<<nboxes, kThreads, smem, st>>>(L, bl, smax, use_smem);
    }
    // spread big pair blocks over several blocks when the colour has few boxes (output tiles of 64,
    // or 32 for the double-float products)
    const int tw = L.gemm_dfl ? 32 : 64;
    const int tiles = ((L.nmax + tw - 1) / tw) * ((L.nmax + tw - 1) / tw);
    const int nd = L.nd, npair = nd * nd, nact = L.dim == 3 ? 343 : 49;   // active pairs, roughly
    const bool df = std::is_same<T, double>::value && L.gemm_dfl;
    const tune::Key kp{0, df ? 1 : 0, tune::ceil_log2(L.nmax), tune::ceil_log2(nboxes)};
    const tune::Key ks{1, df ? 1 : 0, tune::ceil_log2(L.nmax), tune::ceil_log2(nboxes)};
    const int zs = tune::split(ks, std::max(1, std::min(tiles, (608 + nboxes * nact - 1) / (nboxes * nact))));
    const int zp = tune::split(
        kp, std::max(1, std::min(((smax + tw - 1) / tw) * ((L.nmax + tw - 1) / tw), (608 + nboxes * 8 - 1) / (nboxes * 8))));
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};   // panel start / end, Schur start / end
    bool rec;
    {
        std::lock_guard<std::mutex> lk(tune::mu);
        rec = tune::recording;
    }
    if (rec)
        for (auto& e : tev) cudaEventCreate(&e);
    if (rec) cudaEventRecord(tev[0], st);
    if (ev) cudaEventRecord(ev[1], st);
    if (df) k_panel<T, true><<<dim3(nboxes, nd, zp), kThreads, 0, st>>>(L, bl, colour);
    else k_panel<T, false><<<dim3(nboxes, nd, zp), kThreads, 0, st>>>(L, bl, colour);
    if (ev) cudaEventRecord(ev[2], st);
    if (rec) {
        cudaEventRecord(tev[1], st);
        cudaEventRecord(tev[2], st);
    }
    if (df && L.gemm_tc) {
        // tensor-core products: output tiles of 128 x 32, 82.6 KB of dynamic shared memory
        static std::atomic<bool> tc_attr{false};
        if (!tc_attr.load()) {
            cudaFuncSetAttribute(k_schur<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
            tc_attr.store(true);
        }
        const int ttiles = ((L.nmax + tc::kTM - 1) / tc::kTM) * ((L.nmax + tc::kTN - 1) / tc::kTN);
        const int zt = std::max(1, std::min(ttiles, (608 + nboxes * nact - 1) / (nboxes * nact)));
        k_schur<T, 2><<<dim3(nboxes, npair, zt), tc::kThreads, tc::kSmemBytes, st>>>(L, bl, colour);
    } else if (df) {
        k_schur<T, 1><<<dim3(nboxes, npair, zs), kThreads, 0, st>>>(L, bl, colour);
    } else {
        k_schur<T, 0><<<dim3(nboxes, npair, zs), kThreads, 0, st>>>(L, bl, colour);
    }
    if (ev) cudaEventRecord(ev[3], st);
    if (rec) {
        cudaEventRecord(tev[3], st);
        std::lock_guard<std::mutex> lk(tune::mu);
        tune::recs.push_back({kp, tev[0], tev[1]});
        tune::recs.push_back({ks, tev[2], tev[3]});
    }
    // u holds a neighbour's n_q rows (sized by the level bound, not by this colour's pivots), then
    // 8 x RC coefficients, then the column norms of the stacked fill (at most 2 x 5 partners x nmax
    // in 2D, 2 x 19 in 3D)
    // arrays above 64 KB go to the colour's global scratch (read through L1 / L2) so that wide fills
    // neither fail nor cut the number of resident blocks
    size_t csmem = (size_t)(smax_bound + 8 * L.RC + (L.dim == 3 ? 38 : 10) * L.nmax) * sizeof(double);
    const int gscr = (csmem > (size_t)64 * 1024 || !L.Cws) ? 1 : 0;
    // few boxes (the upper levels): one cluster of Cc blocks per compression, each block a slice of
    // the fill's columns, so that the colour's few compressions occupy more SMs; the work arrays of
    // a block (u, coefficients, the norms of its columns, u again) then fit in shared memory
    int Cc = 1;
    const int cmax = compress_cluster_max.load();
    while (Cc < cmax && (size_t)nboxes * (nd - 1) / 2 * Cc < (size_t)2 * num_sms()) Cc *= 2;
    const size_t mbound = (size_t)(L.symmetric ? (L.dim == 3 ? 19 : 5) : (L.dim == 3 ? 38 : 10)) * L.nmax;
    auto cl_smem = [&](int cc) {
        return (size_t)(smax_bound + 8 * L.RC + (mbound + cc - 1) / cc + L.nmax) * sizeof(double);
    };
    while (Cc > 1 && cl_smem(Cc) > (size_t)dynamic_smem_limit(df ? (const void*)k_compress<T, true>
                                                                      : (const void*)k_compress<T, false>))
        Cc = 1;
    bool launched = false;
    for (; Cc > 1 && !launched; Cc = Cc > 8 ? 8 : 1) {
        launched = df ? launch_clustered(k_compress<T, true>, Cc, dim3((unsigned)(nboxes * Cc), (unsigned)nd),
                                         cl_smem(Cc), st, L, bl, colour, 0, Cc)
                      : launch_clustered(k_compress<T, false>, Cc, dim3((unsigned)(nboxes * Cc), (unsigned)nd),
                                         cl_smem(Cc), st, L, bl, colour, 0, Cc);
        if (launched) break;
    }
    if (launched) {
        // one compression per cluster
    } else if (gscr && !L.Cws) {
        k_set_flag<<<1, 1, 0, st>>>(L.status, DEV_ERR_SIZE);   // no scratch was provided: refuse
        count_launches(1);
    } else if (df) {
        k_compress<T, true><<<dim3(nboxes, nd), kThreads, gscr ? 0 : csmem, st>>>(L, bl, colour, gscr, 1);
    } else {
        k_compress<T, false><<<dim3(nboxes, nd), kThreads, gscr ? 0 : csmem, st>>>(L, bl, colour, gscr, 1);
    }
    if (ev) cudaEventRecord(ev[4], st);
    if (df) k_redirect<T, true><<<dim3(nboxes, npair), kThreads, 0, st>>>(L, bl, colour);
    else k_redirect<T, false><<<dim3(nboxes, npair), kThreads, 0, st>>>(L, bl, colour);
    if (ev) cudaEventRecord(ev[5], st);
    count_launches(5);
}

// ---------------------------------------------------------------------------------------------
// level set-up: leaf P2P, or the non-leaf P2P from the children's M2L (Remark in Section 4.2:
// P2P_ij^(k) = [M2L_{i_a j_b}^(k+1)]); W from the orthonormalised operators; initial M2L
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_init_p2p_leaf(LevelView<T> L, const double* p2p0, const int64_t* p2p0_off) {
    const int b = blockIdx.x, d = blockIdx.y;
    const Cell cq = cell_dir(cell_of(b, L.side, L.dim), d, L.dim);
    if (!cell_in(cq, L.side)) return;
    const int q = cell_index(cq, L.side);
    int ld;
    T* dst = block_at(L, b, q, ld);
    const double* src = p2p0 + p2p0_off[(int64_t)b * L.nd + d];
    const int nb_ = L.n[b], nq = L.n[q];
    for (int t = threadIdx.x; t < nb_ * nq; t += blockDim.x) {
        int i = t / nq, j = t - i * nq;
        dst[(size_t)i * ld + j] = (T)src[(size_t)i * nq + j];
    }
}

template <typename T>
__global__ void k_init_p2p_parent(LevelView<T> L, LevelView<T> C, const int* xoff) {
    // blockIdx.y = (direction, child a of b, child bb of q); 2^d children, 2^d + 1 offsets per box
    const int nk = 1 << L.dim, nk2 = nk * nk;
    const int b = blockIdx.x, d = blockIdx.y / nk2, ab = blockIdx.y % nk2;
    const int a = ab / nk, bb = ab % nk;
    const Cell cb = cell_of(b, L.side, L.dim);
    const Cell cq = cell_dir(cb, d, L.dim);
    if (!cell_in(cq, L.side)) return;
    const int q = cell_index(cq, L.side);
    const int ca = cell_index(child_cell(cb, a), C.side);
    const int db = cell_index(child_cell(cq, bb), C.side);
    int lds;
    const T* src = block_at(C, ca, db, lds);
    if (!src) return;
    int ld;
    T* dst = block_at(L, b, q, ld);
    const int ro = xoff[b * (nk + 1) + a], co = xoff[q * (nk + 1) + bb];
    const int rr = C.r[ca], rc = C.r[db];
    for (int t = threadIdx.x; t < rr * rc; t += blockDim.x) {
        int i = t / rc, j = t - i * rc;
        dst[(size_t)(ro + i) * ld + co + j] = src[(size_t)i * lds + j];
    }
}

template <typename T>
__global__ void k_init_far(LevelView<T> L, const double* far0, const int* rank0, int r0) {
    const int b = blockIdx.x, j = blockIdx.y;
    const Cell cb = cell_of(b, L.side, L.dim);
    const Cell cq = region_cell(cb, j, L.dim);
    if (!cell_in(cq, L.side)) return;
    if (cheb_dist(cq, cb) <= 1) return;
    const int q = cell_index(cq, L.side);
    const int64_t o = L.boff[(int64_t)b * L.nreg + j];
    if (o < 0) return;
    T* dst = L.blk + o;
    const int ld = L.bld[(int64_t)b * L.nreg + j];
    const double* src = far0 + ((int64_t)b * L.nreg + j) * r0 * r0;
    const int rb = rank0[b], rq = rank0[q];
    for (int t = threadIdx.x; t < rb * rq; t += blockDim.x) {
        int i = t / rq, jj = t - i * rq;
        dst[(size_t)i * ld + jj] = (T)src[(size_t)i * r0 + jj];
    }
}

template <typename T>
__global__ void k_init_w(LevelView<T> L, int is_leaf, const double* W0, const int64_t* w0_rowoff, int r0,
                         const int* xoff, const int* rank_child, int child_side) {
    const int b = blockIdx.x;
    const int RC = L.RC;
    T* W = L.W + L.voff[b] * RC;
    const int rb = L.r[b];
    if (is_leaf) {
        const double* src = W0 + w0_rowoff[b] * r0;
        const int n = L.n[b];
        for (int t = threadIdx.x; t < n * rb; t += blockDim.x) {
            int i = t / rb, j = t - i * rb;
            W[(size_t)i * RC + j] = (T)src[(size_t)i * r0 + j];
        }
    } else {
        const int nk = 1 << L.dim;
        const double* src = W0 + (int64_t)b * nk * r0 * r0;
        const Cell cb = cell_of(b, L.side, L.dim);
        for (int c = 0; c < nk; ++c) {
            const int cg = cell_index(child_cell(cb, c), child_side);
            const int rc = rank_child[cg];
            const int ro = xoff[b * (nk + 1) + c];
            for (int t = threadIdx.x; t < rc * rb; t += blockDim.x) {
                int i = t / rb, j = t - i * rb;
                W[(size_t)(ro + i) * RC + j] = (T)src[(size_t)(c * r0 + i) * r0 + j];
            }
        }
    }
}

template <typename T>
void launch_init_level(const LevelView<T>& L, int is_leaf, const double* p2p0, const int64_t* p2p0_off,
                       const double* W0, const int64_t* w0_rowoff, int r0, const int* xoff,
                       const double* far0, const int* rank0, const int* rank0_child, const LevelView<T>* child,
                       cudaStream_t st) {
    const int nk = 1 << L.dim;
    if (is_leaf) {
        k_init_p2p_leaf<T><<<dim3(L.nb, L.nd), kThreads, 0, st>>>(L, p2p0, p2p0_off);
    } else {
        k_init_p2p_parent<T><<<dim3(L.nb, L.nd * nk * nk), kThreads, 0, st>>>(L, *child, xoff);
    }
    k_init_far<T><<<dim3(L.nb, L.nreg), kThreads, 0, st>>>(L, far0, rank0, r0);
    k_init_w<T><<<L.nb, kThreads, 0, st>>>(L, is_leaf, W0, w0_rowoff, r0, xoff, rank0_child,
                                           is_leaf ? 0 : child->side);
    count_launches(3);
}

// largest column norm over the diagonal blocks P2P_bb of the level (threshold reference, tau_ref = 1)
template <typename T>
__global__ void k_level_scale(LevelView<T> L, unsigned long long* out) {
    const int b = blockIdx.x;
    int ld;
    const T* D = block_at(L, b, b, ld);
    const int n = L.n[b];
    double mx = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            double v = (double)D[(size_t)i * ld + j];
            s += v * v;
        }
        mx = fmax(mx, sqrt(s));
    }
    if (mx > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

template <typename T>
void launch_level_scale(const LevelView<T>& L, double* out, cudaStream_t st) {
    k_level_scale<T><<<L.nb, 128, 0, st>>>(L, reinterpret_cast<unsigned long long*>(out));
    count_launches(1);
}

// ---------------------------------------------------------------------------------------------
// level 1: the level-2 multipoles as unknowns, P2P^(1) = [M2L^(2)_{cd}] dense
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_root_gather(LevelView<T> L2, const int64_t* rootoff, double* D, int M) {
    const int b = blockIdx.x, q = blockIdx.y;
    int ld;
    const T* src = block_at(L2, b, q, ld);
    if (!src) return;
    const int rb = L2.r[b], rq = L2.r[q];
    const int64_t ro = rootoff[b], co = rootoff[q];
    for (int t = threadIdx.x; t < rb * rq; t += blockDim.x) {
        int i = t / rq, j = t - i * rq;
        D[(ro + i) * M + co + j] = (double)src[(size_t)i * ld + j];
    }
}

template <typename T>
void launch_root_gather(const LevelView<T>& L2, const int64_t* rootoff, double* D, int M, cudaStream_t st) {
    k_root_gather<T><<<dim3(L2.nb, L2.nb), kThreads, 0, st>>>(L2, rootoff, D, M);
    count_launches(1);
}

__global__ void __launch_bounds__(1024) k_dense_invert(double* D, int M, int* perm, double* col, int* status) {
    __shared__ double vred[32];
    __shared__ int ired[32];
    bool ok = cta_gauss_jordan(D, M, M, perm, col, vred, ired);
    if (!ok && threadIdx.x == 0) atomicOr(status, DEV_ERR_SINGULAR);
}

// The same Gauss-Jordan elimination spread over the GPU for large M, two launches per column: the
// pivot step (one block: partial pivoting with ties to the lowest row, row interchange, scaling of
// the pivot row, copy of the pivot column) and the update of every other row (one block per row
// and 256 columns). Every element sees the operations of cta_gauss_jordan in the same order.
// perm[M] is the failure flag (set on a zero or non-finite pivot; later launches then return),
// col[M] keeps 1 / pivot for the update.
__global__ void __launch_bounds__(1024) k_gj_pivot(double* A, int M, int k, int* perm, double* col, int* status) {
    __shared__ double vred[32];
    __shared__ int ired[32];
    __shared__ int s_ok;
    __shared__ double s_piv;
    if (perm[M]) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    double best = -1.0;
    int bi = -1;
    for (int i = k + tid; i < M; i += nt) {
        const double v = fabs(A[(size_t)i * M + k]);
        if (bi < 0 || v > best) { best = v; bi = i; }
    }
    double bv;
    const int p = block_argmax(best, bi, vred, ired, &bv);
    if (tid == 0) {
        perm[k] = p;
        s_ok = (p >= 0 && bv > 0.0 && isfinite(bv)) ? 1 : 0;
        if (!s_ok) {
            perm[M] = 1;
            atomicOr(status, DEV_ERR_SINGULAR);
        }
    }
    __syncthreads();
    if (!s_ok) return;
    if (p != k)
        for (int j = tid; j < M; j += nt) {
            const double t = A[(size_t)k * M + j];
            A[(size_t)k * M + j] = A[(size_t)p * M + j];
            A[(size_t)p * M + j] = t;
        }
    __syncthreads();
    if (tid == 0) s_piv = A[(size_t)k * M + k];
    __syncthreads();
    const double d = 1.0 / s_piv;
    for (int j = tid; j < M; j += nt) {
        if (j == k) A[(size_t)k * M + k] = d;
        else A[(size_t)k * M + j] *= d;
    }
    for (int i = tid; i < M; i += nt) col[i] = i == k ? d : A[(size_t)i * M + k];
    if (tid == 0) col[M] = d;
}

__global__ void __launch_bounds__(256) k_gj_update(double* A, int M, int k, const int* perm, const double* col) {
    if (perm[M]) return;
    const int i = blockIdx.y, j = blockIdx.x * 256 + threadIdx.x;
    if (i == k || j >= M) return;
    const double c = col[i];
    if (j == k) A[(size_t)i * M + k] = -c * col[M];
    else A[(size_t)i * M + j] -= c * A[(size_t)k * M + j];
}

// undo the row interchanges as column interchanges, last first: row-local, one thread per row
__global__ void __launch_bounds__(256) k_gj_unswap(double* A, int M, const int* perm) {
    if (perm[M]) return;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= M) return;
    double* row = A + (size_t)i * M;
    for (int k = M - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k) {
            const double t = row[k];
            row[k] = row[p];
            row[p] = t;
        }
    }
}

// perm: M + 1 ints, col: M + 1 doubles of scratch
void launch_dense_invert(double* D, int M, int* perm, double* col, int* status, cudaStream_t st) {
    if (M <= 0) return;
    if (M < 256 || M > 65535) {   // one block: fewer launches than the per-column steps cost (or
                                   // more rows than a grid dimension holds)
        k_dense_invert<<<1, 1024, 0, st>>>(D, M, perm, col, status);
        count_launches(1);
        return;
    }
    cudaMemsetAsync(perm + M, 0, sizeof(int), st);
    const dim3 ug((M + 255) / 256, M);
    for (int k = 0; k < M; ++k) {
        k_gj_pivot<<<1, 1024, 0, st>>>(D, M, k, perm, col, status);
        k_gj_update<<<ug, 256, 0, st>>>(D, M, k, perm, col);
    }
    k_gj_unswap<<<(M + 255) / 256, 256, 0, st>>>(D, M, perm);
    count_launches(2 * M + 1);
}

template <typename T>
__global__ void k_root_apply(const double* Dinv, int M, const T* rhs, T* x, int nrhs) {
    __shared__ double sm[gemm_smem<double>::value];
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    const int mm = min(64, M - m0), nn = min(64, nrhs - n0);
    cta_gemm<double>(
        mm, nn, M, [&](int i, int k) { return Dinv[(size_t)(m0 + i) * M + k]; },
        [&](int k, int j) { return (double)rhs[(size_t)k * nrhs + n0 + j]; },
        [&](int i, int j, double v) { x[(size_t)(m0 + i) * nrhs + n0 + j] = (T)v; }, sm);
}

template <typename T>
void launch_root_apply(const double* Dinv, int M, const T* rhs, T* x, int nrhs, cudaStream_t st) {
    if (M <= 0) return;
    k_root_apply<T><<<dim3((M + 63) / 64, (nrhs + 63) / 64), kThreads, 0, st>>>(Dinv, M, rhs, x, nrhs);
    count_launches(1);
}

// ---------------------------------------------------------------------------------------------
// replay: forward over the stored factors, back substitution (Algorithm 2)
// ---------------------------------------------------------------------------------------------
// The replay's products in the working precision (a CTA GEMM); the tensor-core replay (FP64
// vectors, factors split once into digit slabs) is the k_*_slab family below
template <int GM>
struct ReplayGemm;
template <>
struct ReplayGemm<0> {
    template <typename T, class LA, class LB, class EPI>
    static IFMM_DEVINL void run(int M, int N, int K, LA la, LB lb, EPI epi, void* sm, int* status, int tile0,
                                int tstride) {
        using Acc = typename AccOf<T>::type;
        (void)status;
        cta_gemm<Acc>(M, N, K, la, lb, epi, (Acc*)sm, tile0, tstride);
    }
};
// shared memory of a replay CTA: the CTA GEMM's tiles (GM = 0) or the dynamic tensor-core tiles
template <typename T, int GM>
struct ReplaySmem {
    using Acc = typename AccOf<T>::type;
    static constexpr int elems = GM == 2 ? 1 : gemm_smem<Acc>::value;
};
#define IFMM_REPLAY_SMEM(T, GM)                                                            \
    __shared__ typename AccOf<T>::type rsm_static[ReplaySmem<T, GM>::elems];               \
    extern __shared__ __align__(1024) uint8_t rsm_dyn[];                                   \
    void* rsm = GM == 2 ? (void*)rsm_dyn : (void*)rsm_static;
// output tile of the replay GEMM (rows x columns) for the split-K reduction
template <typename T, int GM>
struct ReplayTile {
    static constexpr int M = GM == 2 ? tc::kTM : (std::is_same<T, dfl>::value ? 32 : 64);
    static constexpr int N = GM == 2 ? tc::kTN : (std::is_same<T, dfl>::value ? 32 : 64);
};

// ---- the tensor-core replay: factors from their digit slabs, vectors split per block -------------
IFMM_DEVINL int active_width_at(const int* n, const int* r, int side, int q, int colour_e) {
    const int qx = q % side, qy = q / side;
    return colour_of(qx, qy) < colour_e ? r[q] : n[q];
}

// one record's slab and row exponents
IFMM_DEVINL const uint8_t* slab_of(const SlabSet& S, int e, int rec) {
    return S.slab + S.soff[(int64_t)e * kSlabRecs + rec];
}
IFMM_DEVINL const int* rexp_of(const SlabSet& S, int e, int rec) { return S.rexp + S.eoff[(int64_t)e * kSlabRecs + rec]; }

__global__ void __launch_bounds__(tc::kSlabThreads) k_presplit(LevelView<double> L, uint8_t* slab, int* rexp,
                                                               const int* boxes, int colour) {
    const int e = boxes[blockIdx.x];
    const int rec = blockIdx.y;
    const int64_t so = L.sl.soff[(int64_t)e * kSlabRecs + rec];
    if (so < 0) return;
    uint8_t* sp = slab + so;
    int* ep = rexp + L.sl.eoff[(int64_t)e * kSlabRecs + rec];
    const int n = L.n[e], r = L.r[e], s = n + r;
    const int ex = e % L.side, ey = e / L.side;
    const double* Pi = L.Pi + L.pioff[e];
    const int ld = L.pild[e];
    if (rec == 0) {
        tc::split_to_slab(s, n, [&](int i, int k) { return Pi[(size_t)i * ld + k]; }, sp, ep);
    } else if (rec == 1) {
        tc::split_to_slab(n, s, [&](int i, int k) { return Pi[(size_t)i * ld + k]; }, sp, ep);
    } else if (rec < 11) {
        const int d = rec - 2;
        const int q = (ex + d % 3 - 1) + L.side * (ey + d / 3 - 1);
        const int w = active_width_at(L.n, L.r, L.side, q, colour);
        const double* C = L.Cp + L.cpoff[(int64_t)e * 9 + d];
        tc::split_to_slab(w, n, [&](int i, int k) { return C[(size_t)i * n + k]; }, sp, ep);
    } else {
        __shared__ const double* sB[8];
        __shared__ int sOff[9], sW[8];
        if (threadIdx.x == 0) {
            int c = 0, off = 0;
            for (int d = 0; d < 9; ++d) {
                if (d == 4) continue;
                const int qx = ex + d % 3 - 1, qy = ey + d / 3 - 1;
                if (!in_grid(qx, qy, L.side)) continue;
                const int q = qx + L.side * qy;
                sB[c] = L.Bp + L.bpoff[(int64_t)e * 9 + d];
                sW[c] = active_width_at(L.n, L.r, L.side, q, colour);
                sOff[c] = off;
                off += sW[c];
                ++c;
            }
            for (int t = c; t < 9; ++t) sOff[t] = off;
        }
        __syncthreads();
        const int K = sOff[8];
        tc::split_to_slab(n, K, [&](int i, int k) {
            int c = 0;
            while (c < 7 && k >= sOff[c + 1]) ++c;
            return sB[c][(size_t)i * sW[c] + (k - sOff[c])];
        }, sp, ep);
    }
}

void launch_presplit(const LevelView<double>& L, uint8_t* slab, int* rexp, const int* boxes, int nboxes, int colour,
                     cudaStream_t st) {
    if (nboxes <= 0) return;
    k_presplit<<<dim3(nboxes, kSlabRecs), tc::kSlabThreads, 0, st>>>(L, slab, rexp, boxes, colour);
    count_launches(1);
}

IFMM_DEVINL int slab_rg(int rows) { return (rows + 7) / 8; }

// The slab kernels are persistent: a grid of at most two blocks per SM walks the items (box, tile
// group) of the launch, with tensor memory and the mbarrier set up once per block.
__global__ void __launch_bounds__(tc::kSlabThreads, 2) k_fwd_piv_slab(LevelView<double> L, const int* boxes,
                                                                     int nboxes, int Z, const int64_t* yoff,
                                                                     double* vec_k, double* vec_km1, double* vx,
                                                                     int nrhs) {
    extern __shared__ __align__(1024) uint8_t tsm[];
    tc::Ctx c;
    tc::ctx_init(c, tsm, L.status);
    for (int item = blockIdx.x; item < nboxes * Z; item += gridDim.x) {
        const int e = boxes[item / Z], z = item % Z;
        const int n = L.n[e], r = L.r[e], s = n + r;
        if (s == 0) continue;
        const double* rhs = vec_k + L.voff[e] * nrhs;
        double* vxe = vx + L.voff[e] * nrhs;
        double* ze = vec_km1 + yoff[e] * nrhs;
        // v = Pi [rhs_e; 0]: x rows to vx, z rows become the M2L_e right-hand side
        tc::tc_gemm_slab(
            c, slab_of(L.sl, e, 0), rexp_of(L.sl, e, 0), slab_rg(s), 0, s, nrhs, n,
            [&](int k, int j) { return rhs[(size_t)k * nrhs + j]; },
            [&](int i, int j, double v) {
                if (i < n) vxe[(size_t)i * nrhs + j] = v;
                else ze[(size_t)(i - n) * nrhs + j] = v;
            },
            z, Z);
    }
    tc::ctx_release(c);
}

__global__ void __launch_bounds__(tc::kSlabThreads, 2) k_fwd_upd_slab(LevelView<double> L, const int* boxes,
                                                                     int nboxes, int Z, int colour,
                                                                     const int64_t* yoff, double* vec_k,
                                                                     double* vec_km1, const double* vx, int nrhs) {
    extern __shared__ __align__(1024) uint8_t tsm[];
    tc::Ctx c;
    tc::ctx_init(c, tsm, L.status);
    for (int item = blockIdx.x; item < nboxes * 8 * Z; item += gridDim.x) {
        const int e = boxes[item / (8 * Z)];
        const int dd = (item / Z) % 8, z = item % Z;
        const int dp = dd < 4 ? dd : dd + 1;      // neighbour directions without 4 (e itself)
        const int ex = e % L.side, ey = e / L.side;
        const int px = ex + dp % 3 - 1, py = ey + dp / 3 - 1;
        if (!in_grid(px, py, L.side)) continue;
        const int p = px + L.side * py;
        const bool Ep = colour_of(px, py) < colour;
        const int wp = Ep ? L.r[p] : L.n[p];
        const int n = L.n[e];
        if (wp == 0 || n == 0) continue;
        const double* v = vx + L.voff[e] * nrhs;
        double* tgt = Ep ? vec_km1 + yoff[p] * nrhs : vec_k + L.voff[p] * nrhs;
        tc::tc_gemm_slab(
            c, slab_of(L.sl, e, 2 + dp), rexp_of(L.sl, e, 2 + dp), slab_rg(wp), 0, wp, nrhs, n,
            [&](int k, int j) { return v[(size_t)k * nrhs + j]; },
            [&](int i, int j, double a) { tgt[(size_t)i * nrhs + j] -= a; }, z, Z);
    }
    tc::ctx_release(c);
}

// back substitution, first half, from the slab of the side-by-side B panels; split-K as k_bwd_w
// (item = box x (tile group tg of zt + zt x K split kz of ks))
__global__ void __launch_bounds__(tc::kSlabThreads, 2) k_bwd_w_slab(LevelView<double> L, const int* boxes,
                                                                   int nboxes, int colour, const int64_t* yoff,
                                                                   const double* rhs_k, const double* x_k,
                                                                   const double* x_km1, double* wtmp, int nrhs,
                                                                   int zt, int ks, double* part, int* cnt,
                                                                   int64_t pstride) {
    extern __shared__ __align__(1024) uint8_t tsm[];
    __shared__ const double* sU[8];
    __shared__ int sOff[9];
    __shared__ int s_last;
    tc::Ctx c;
    tc::ctx_init(c, tsm, L.status);
    const int per = zt * ks;
    constexpr int TM = tc::kTM, TN = tc::kTN;
    const int tn = (nrhs + TN - 1) / TN;
    for (int item = blockIdx.x; item < nboxes * per; item += gridDim.x) {
        const int bi = item / per, zz = item % per;
        const int e = boxes[bi];
        const int ex = e % L.side, ey = e / L.side;
        const int n = L.n[e];
        const int tg = zz % zt, kz = zz / zt;
        __syncthreads();   // the previous item's readers of sU / sOff are done
        if (threadIdx.x == 0) {
            int cc = 0, off = 0;
            for (int d = 0; d < 9; ++d) {
                if (d == 4) continue;
                const int qx = ex + d % 3 - 1, qy = ey + d / 3 - 1;
                if (!in_grid(qx, qy, L.side)) continue;
                const int q = qx + L.side * qy;
                const bool Eq = colour_of(qx, qy) < colour;
                sU[cc] = Eq ? x_km1 + yoff[q] * nrhs : x_k + L.voff[q] * nrhs;
                sOff[cc] = off;
                off += Eq ? L.r[q] : L.n[q];
                ++cc;
            }
            for (int t = cc; t < 9; ++t) sOff[t] = off;
        }
        __syncthreads();
        if (n == 0) continue;
        const int K = sOff[8];
        auto lb = [&](int k, int j) {
            int cc = 0;
            while (cc < 7 && k >= sOff[cc + 1]) ++cc;
            return sU[cc][(size_t)(k - sOff[cc]) * nrhs + j];
        };
        double* w = wtmp + L.voff[e] * nrhs;
        const double* rhs = rhs_k + L.voff[e] * nrhs;
        const uint8_t* sp = slab_of(L.sl, e, 11);
        const int* ep = rexp_of(L.sl, e, 11);
        if (ks == 1) {
            if (K == 0) {
                for (int t = threadIdx.x + tg * blockDim.x; t < n * nrhs; t += blockDim.x * zt) w[t] = rhs[t];
                continue;
            }
            tc::tc_gemm_slab(c, sp, ep, slab_rg(n), 0, n, nrhs, K, lb,
                             [&](int i, int j, double a) { w[(size_t)i * nrhs + j] = rhs[(size_t)i * nrhs + j] - a; },
                             tg, zt);
            continue;
        }
        const int chunk = (((K + ks - 1) / ks) + 31) & ~31;
        const int k_lo = min(K, kz * chunk), k_hi = min(K, k_lo + chunk);
        double* P = part + ((int64_t)kz * nboxes + bi) * pstride;
        if (k_hi > k_lo) {
            tc::tc_gemm_slab(c, sp, ep, slab_rg(n), k_lo / tc::kKC, n, nrhs, k_hi - k_lo,
                             [&](int k, int j) { return lb(k_lo + k, j); },
                             [&](int i, int j, double a) { P[(size_t)i * nrhs + j] = a; }, tg, zt);
        } else {
            for (int t = threadIdx.x; t < n * nrhs; t += blockDim.x) {
                const int i = t / nrhs, j = t - i * nrhs;
                if (((i / TM) * tn + j / TN) % zt == tg) P[(size_t)i * nrhs + j] = 0.0;
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(&cnt[bi * zt + tg], 1) == ks - 1) ? 1 : 0;
        __syncthreads();
        if (!s_last) continue;
        __threadfence();
        for (int t = threadIdx.x; t < n * nrhs; t += blockDim.x) {
            const int i = t / nrhs, j = t - i * nrhs;
            if (((i / TM) * tn + j / TN) % zt != tg) continue;
            double a = 0.0;
            for (int z = 0; z < ks; ++z) a += __ldcg(part + ((int64_t)z * nboxes + bi) * pstride + (size_t)i * nrhs + j);
            w[(size_t)i * nrhs + j] = rhs[(size_t)i * nrhs + j] - a;
        }
        if (threadIdx.x == 0) cnt[bi * zt + tg] = 0;
    }
    tc::ctx_release(c);
}

// back substitution, second half: [x_e; z_e] = Pi [w; y_e] from the slab of Pi's first n rows
__global__ void __launch_bounds__(tc::kSlabThreads, 2) k_bwd_x_slab(LevelView<double> L, const int* boxes,
                                                                   int nboxes, int Z, const int64_t* yoff,
                                                                   double* x_k, const double* x_km1,
                                                                   const double* wtmp, int nrhs) {
    extern __shared__ __align__(1024) uint8_t tsm[];
    tc::Ctx c;
    tc::ctx_init(c, tsm, L.status);
    for (int item = blockIdx.x; item < nboxes * Z; item += gridDim.x) {
        const int e = boxes[item / Z], z = item % Z;
        const int n = L.n[e], r = L.r[e], s = n + r;
        if (n == 0) continue;
        const double* w = wtmp + L.voff[e] * nrhs;
        const double* ye = x_km1 + yoff[e] * nrhs;
        double* xe = x_k + L.voff[e] * nrhs;
        tc::tc_gemm_slab(
            c, slab_of(L.sl, e, 1), rexp_of(L.sl, e, 1), slab_rg(n), 0, n, nrhs, s,
            [&](int k, int j) { return k < n ? w[(size_t)k * nrhs + j] : ye[(size_t)(k - n) * nrhs + j]; },
            [&](int i, int j, double a) { xe[(size_t)i * nrhs + j] = a; }, z, Z);
    }
    tc::ctx_release(c);
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cudaGetLastError();
        sms = v;
    }
    return sms;
}

void set_slab_smem() {
    static std::atomic<bool> done{false};
    if (done.load()) return;
    cudaFuncSetAttribute(k_fwd_piv_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
    cudaFuncSetAttribute(k_fwd_upd_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
    cudaFuncSetAttribute(k_bwd_w_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
    cudaFuncSetAttribute(k_bwd_x_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
    done.store(true);
}

template <typename T, int GM>
__global__ void __launch_bounds__(GM == 2 ? tc::kThreads : kThreads) k_fwd_piv(LevelView<T> L, const int* boxes,
                                                                              const int64_t* yoff, T* vec_k,
                                                                              T* vec_km1, T* vx, int nrhs) {
    using Acc = typename AccOf<T>::type;
    IFMM_REPLAY_SMEM(T, GM)
    const int e = boxes[blockIdx.x];
    const int n = L.n[e], r = L.r[e], s = n + r;
    const T* Pi = L.Pi + L.pioff[e];
    const int ld = L.pild[e];
    const T* rhs = vec_k + L.voff[e] * nrhs;
    T* vxe = vx + L.voff[e] * nrhs;
    T* ze = vec_km1 + yoff[e] * nrhs;
    if (s == 0) return;
    // v = Pi [rhs_e; 0]: x rows to vx, z rows become the M2L_e right-hand side
    ReplayGemm<GM>::template run<T>(
        s, nrhs, n, [&](int i, int k) { return Pi[(size_t)i * ld + k]; },
        [&](int k, int j) { return rhs[(size_t)k * nrhs + j]; },
        [&](int i, int j, Acc v) {
            if (i < n) vxe[(size_t)i * nrhs + j] = (T)v;
            else ze[(size_t)(i - n) * nrhs + j] = (T)v;
        },
        rsm, L.status, blockIdx.z, gridDim.z);
}

template <typename T, int GM>
__global__ void __launch_bounds__(GM == 2 ? tc::kThreads : kThreads) k_fwd_upd(LevelView<T> L, const int* boxes,
                                                                              int colour, const int64_t* yoff,
                                                                              T* vec_k, T* vec_km1, const T* vx,
                                                                              int nrhs) {
    using Acc = typename AccOf<T>::type;
    IFMM_REPLAY_SMEM(T, GM)
    const int e = boxes[blockIdx.x];
    const int dp = blockIdx.y;
    if (dp == L.ctr) return;
    const Cell cp = cell_dir(cell_of(e, L.side, L.dim), dp, L.dim);
    if (!cell_in(cp, L.side)) return;
    const int p = cell_index(cp, L.side);
    const bool Ep = cell_colour(cp) < colour;
    const int wp = Ep ? L.r[p] : L.n[p];
    const int n = L.n[e];
    if (wp == 0) return;
    const T* C = L.Cp + L.cpoff[(int64_t)e * L.nd + dp];
    const T* v = vx + L.voff[e] * nrhs;
    T* tgt = Ep ? vec_km1 + yoff[p] * nrhs : vec_k + L.voff[p] * nrhs;
    ReplayGemm<GM>::template run<T>(
        wp, nrhs, n, [&](int i, int k) { return C[(size_t)i * n + k]; },
        [&](int k, int j) { return v[(size_t)k * nrhs + j]; },
        [&](int i, int j, Acc a) { tgt[(size_t)i * nrhs + j] = (T)((Acc)tgt[(size_t)i * nrhs + j] - a); }, rsm,
        L.status, blockIdx.z, gridDim.z);
}

template <typename T>
void launch_forward_colour(const LevelView<T>& L, const int* boxes, int nboxes, int colour, const int64_t* yoff,
                           T* vec_k, T* vec_km1, T* vx, int nrhs, cudaStream_t st) {
    if (nboxes <= 0) return;
    const int smax = L.nmax + std::min(L.nmax, L.RC);
    count_launches(2);
    if constexpr (std::is_same<T, double>::value) {
        if (L.sl.slab) {
            constexpr int TM = tc::kTM, TN = tc::kTN;
            const int tr = (nrhs + TN - 1) / TN;
            const int z1 = std::max(1, std::min(((smax + TM - 1) / TM) * tr, (304 + nboxes - 1) / nboxes));
            const int z2 = std::max(1, std::min(((L.nmax + TM - 1) / TM) * tr, (304 + nboxes * 8 - 1) / (nboxes * 8)));
            set_slab_smem();
            const int cap = 2 * num_sms();
            k_fwd_piv_slab<<<std::min(nboxes * z1, cap), tc::kSlabThreads, tc::kSmemBytes, st>>>(
                L, boxes, nboxes, z1, yoff, vec_k, vec_km1, vx, nrhs);
            k_fwd_upd_slab<<<std::min(nboxes * 8 * z2, cap), tc::kSlabThreads, tc::kSmemBytes, st>>>(
                L, boxes, nboxes, z2, colour, yoff, vec_k, vec_km1, vx, nrhs);
            return;
        }
    }
    const int tw = ReplayTile<T, 0>::M, th = ReplayTile<T, 0>::N;   // output tile of the CTA GEMM
    const int tr = (nrhs + th - 1) / th;
    const int z1 = std::max(1, std::min(((smax + tw - 1) / tw) * tr, (608 + nboxes - 1) / nboxes));
    const int nn = L.nd - 1;   // neighbours other than e
    const int z2 = std::max(1, std::min(((L.nmax + tw - 1) / tw) * tr, (608 + nboxes * nn - 1) / (nboxes * nn)));
    k_fwd_piv<T, 0><<<dim3(nboxes, 1, z1), kThreads, 0, st>>>(L, boxes, yoff, vec_k, vec_km1, vx, nrhs);
    k_fwd_upd<T, 0><<<dim3(nboxes, L.nd, z2), kThreads, 0, st>>>(L, boxes, colour, yoff, vec_k, vec_km1, vx, nrhs);
}

// back substitution, first half: w = rhs_e - sum_q B_q u_q as one GEMM over the concatenated
// panels, u_q = x_q (q eliminated after e) or y_q (before)
// L2-coherent load (the partial sums of split-K are written by other CTAs of the same launch)
IFMM_DEVINL double ldcg_v(const double* p) { return __ldcg(p); }
IFMM_DEVINL float ldcg_v(const float* p) { return __ldcg(p); }
IFMM_DEVINL dfl ldcg_v(const dfl* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return dfl(v.x, v.y);
}

// back substitution, first half: w = rhs_e - sum_q B_q u_q as one GEMM over the concatenated
// panels, u_q = x_q (q eliminated after e) or y_q (before). blockIdx.z = tile group tg (of zt) +
// zt * K-split kz (of ks). With ks > 1 each CTA writes the partial product over its slice of K to
// `part`; the last CTA of a tile group (atomic counter) adds the partials in split order, so the
// result does not depend on the CTAs' timing, and resets the counter.
template <typename T, int GM>
__global__ void __launch_bounds__(GM == 2 ? tc::kThreads : kThreads) k_bwd_w(LevelView<T> L, const int* boxes,
                                                                            int colour, const int64_t* yoff,
                                                                            const T* rhs_k, const T* x_k,
                                                                            const T* x_km1, T* wtmp, int nrhs, int zt,
                                                                            int ks, T* part, int* cnt,
                                                                            int64_t pstride) {
    using Acc = typename AccOf<T>::type;
    IFMM_REPLAY_SMEM(T, GM)
    // the neighbours other than e: 8 in 2D, 26 in 3D
    __shared__ const T* sB[26];
    __shared__ const T* sU[26];
    __shared__ int sOff[27], sW[26];
    __shared__ int s_last;
    const int e = boxes[blockIdx.x];
    const Cell ce = cell_of(e, L.side, L.dim);
    const int n = L.n[e];
    const int nn = L.nd - 1;
    const int tg = blockIdx.z % zt, kz = blockIdx.z / zt;
    if (threadIdx.x == 0) {
        int cnt_ = 0, off = 0;
        for (int d = 0; d < L.nd; ++d) {
            if (d == L.ctr) continue;
            const Cell cq = cell_dir(ce, d, L.dim);
            if (!cell_in(cq, L.side)) continue;
            const int q = cell_index(cq, L.side);
            const bool Eq = cell_colour(cq) < colour;
            const int wq = Eq ? L.r[q] : L.n[q];
            sB[cnt_] = L.Bp + L.bpoff[(int64_t)e * L.nd + d];
            sU[cnt_] = Eq ? x_km1 + yoff[q] * nrhs : x_k + L.voff[q] * nrhs;
            sW[cnt_] = wq;
            sOff[cnt_] = off;
            off += wq;
            ++cnt_;
        }
        for (int c = cnt_; c <= nn; ++c) sOff[c] = off;
    }
    __syncthreads();
    const int K = sOff[nn];
    // segment of column k: the number of segment starts sOff[1..nn-1] at or below k (sOff is
    // nondecreasing); unrolled for the quadtree's 8 neighbours
    auto seg = [&](int k) {
        int c = 0;
        if (nn == 8) {
#pragma unroll
            for (int t = 1; t < 8; ++t) c += sOff[t] <= k ? 1 : 0;
        } else {
            for (int t = 1; t < nn; ++t) c += sOff[t] <= k ? 1 : 0;
        }
        return c;
    };
    auto la = [&](int i, int k) {
        const int c = seg(k);
        return sB[c][(size_t)i * sW[c] + (k - sOff[c])];
    };
    auto lb = [&](int k, int j) {
        const int c = seg(k);
        return sU[c][(size_t)(k - sOff[c]) * nrhs + j];
    };
    T* w = wtmp + L.voff[e] * nrhs;
    const T* rhs = rhs_k + L.voff[e] * nrhs;
    if (n == 0) return;
    if (ks == 1) {
        if (K == 0) {
            for (int t = threadIdx.x + tg * blockDim.x; t < n * nrhs; t += blockDim.x * zt) w[t] = rhs[t];
            return;
        }
        ReplayGemm<GM>::template run<T>(
            n, nrhs, K, la, lb,
            [&](int i, int j, Acc a) { w[(size_t)i * nrhs + j] = (T)((Acc)rhs[(size_t)i * nrhs + j] - a); }, rsm,
            L.status, tg, zt);
        return;
    }
    // this split's slice of K (a multiple of 32 long; possibly empty)
    const int chunk = (((K + ks - 1) / ks) + 31) & ~31;
    const int k_lo = min(K, kz * chunk), k_hi = min(K, k_lo + chunk);
    T* P = part + ((int64_t)kz * gridDim.x + blockIdx.x) * pstride;
    if (k_hi > k_lo) {
        ReplayGemm<GM>::template run<T>(
            n, nrhs, k_hi - k_lo, [&](int i, int k) { return la(i, k_lo + k); },
            [&](int k, int j) { return lb(k_lo + k, j); },
            [&](int i, int j, Acc a) { P[(size_t)i * nrhs + j] = (T)a; }, rsm, L.status, tg, zt);
    } else {
        // an empty slice contributes zeros to the outputs of this tile group
        constexpr int TM = ReplayTile<T, GM>::M, TN = ReplayTile<T, GM>::N;
        const int tn = (nrhs + TN - 1) / TN;
        for (int t = threadIdx.x; t < n * nrhs; t += blockDim.x) {
            const int i = t / nrhs, j = t - i * nrhs;
            if (((i / TM) * tn + j / TN) % zt == tg) P[(size_t)i * nrhs + j] = (T)0;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&cnt[blockIdx.x * zt + tg], 1) == ks - 1) ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // outputs of this tile group (the tiles of the product above)
    constexpr int TM = ReplayTile<T, GM>::M, TN = ReplayTile<T, GM>::N;
    const int tn = (nrhs + TN - 1) / TN;
    for (int t = threadIdx.x; t < n * nrhs; t += blockDim.x) {
        const int i = t / nrhs, j = t - i * nrhs;
        if (((i / TM) * tn + j / TN) % zt != tg) continue;
        Acc acc = (Acc)0;
        for (int z = 0; z < ks; ++z)
            acc = acc + (Acc)ldcg_v(part + ((int64_t)z * gridDim.x + blockIdx.x) * pstride + (size_t)i * nrhs + j);
        w[(size_t)i * nrhs + j] = (T)((Acc)rhs[(size_t)i * nrhs + j] - acc);
    }
    if (threadIdx.x == 0) cnt[blockIdx.x * zt + tg] = 0;
}

// back substitution, second half: [x_e; z_e] = Pi [w; y_e]; only x_e is kept
template <typename T, int GM>
__global__ void __launch_bounds__(GM == 2 ? tc::kThreads : kThreads) k_bwd_x(LevelView<T> L, const int* boxes,
                                                                            const int64_t* yoff, T* x_k,
                                                                            const T* x_km1, const T* wtmp,
                                                                            int nrhs) {
    using Acc = typename AccOf<T>::type;
    IFMM_REPLAY_SMEM(T, GM)
    const int e = boxes[blockIdx.x];
    const int n = L.n[e], r = L.r[e], s = n + r;
    const T* w = wtmp + L.voff[e] * nrhs;
    const T* Pi = L.Pi + L.pioff[e];
    const int ld = L.pild[e];
    const T* ye = x_km1 + yoff[e] * nrhs;
    T* xe = x_k + L.voff[e] * nrhs;
    if (n == 0) return;
    ReplayGemm<GM>::template run<T>(
        n, nrhs, s, [&](int i, int k) { return Pi[(size_t)i * ld + k]; },
        [&](int k, int j) { return k < n ? w[(size_t)k * nrhs + j] : ye[(size_t)(k - n) * nrhs + j]; },
        [&](int i, int j, Acc a) { xe[(size_t)i * nrhs + j] = (T)a; }, rsm, L.status, blockIdx.z, gridDim.z);
}

template <typename T>
void launch_backward_colour(const LevelView<T>& L, const int* boxes, int nboxes, int colour, const int64_t* yoff,
                            const T* rhs_k, T* x_k, const T* x_km1, T* wtmp, int nrhs, T* part, int64_t part_cap,
                            int* cnt, int cnt_cap, cudaStream_t st) {
    if (nboxes <= 0) return;
    const bool tcm = std::is_same<T, double>::value && L.sl.slab != nullptr;
    const int TM = tcm ? ReplayTile<T, 2>::M : ReplayTile<T, 0>::M;
    const int TN = tcm ? ReplayTile<T, 2>::N : ReplayTile<T, 0>::N;
    const int cap_ctas = tcm ? 304 : 608;
    const int z = std::max(1, std::min(((L.nmax + TM - 1) / TM) * ((nrhs + TN - 1) / TN), (cap_ctas + nboxes - 1) / nboxes));
    // few CTAs (upper levels): split K = sum of the neighbours' widths (<= 8 nmax) over more CTAs
    int ks = 1;
    const int64_t pstride = (int64_t)std::max(L.nmax, 1) * nrhs;
    if (part && cnt && nboxes * z < 304 && nboxes * z <= cnt_cap) {
        ks = std::min(16, (304 + nboxes * z - 1) / (nboxes * z));
        ks = std::min(ks, std::max(1, 8 * L.nmax / 64));
        while (ks > 1 && (int64_t)ks * nboxes * pstride > part_cap) --ks;
    }
    count_launches(2);
    if constexpr (std::is_same<T, double>::value) {
        if (tcm) {
            set_slab_smem();
            const int cap = 2 * num_sms();
            k_bwd_w_slab<<<std::min(nboxes * z * ks, cap), tc::kSlabThreads, tc::kSmemBytes, st>>>(
                L, boxes, nboxes, colour, yoff, rhs_k, x_k, x_km1, wtmp, nrhs, z, ks, part, cnt, pstride);
            k_bwd_x_slab<<<std::min(nboxes * z, cap), tc::kSlabThreads, tc::kSmemBytes, st>>>(
                L, boxes, nboxes, z, yoff, x_k, x_km1, wtmp, nrhs);
            return;
        }
    }
    k_bwd_w<T, 0><<<dim3(nboxes, 1, z * ks), kThreads, 0, st>>>(L, boxes, colour, yoff, rhs_k, x_k, x_km1, wtmp,
                                                                 nrhs, z, ks, part, cnt, pstride);
    k_bwd_x<T, 0><<<dim3(nboxes, 1, z), kThreads, 0, st>>>(L, boxes, yoff, x_k, x_km1, wtmp, nrhs);
}

template <typename T>
__global__ void k_permute_in(const double* b, int64_t ld, int64_t N, int nrhs, const int64_t* perm, T* out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * nrhs) return;
    int64_t i = t / nrhs;
    int j = (int)(t - i * nrhs);
    out[t] = (T)b[perm[i] + (int64_t)j * ld];
}

template <typename T>
void launch_permute_in(const double* b, int64_t ld, int64_t N, int nrhs, const int64_t* perm, T* out,
                       cudaStream_t st) {
    int64_t tot = N * nrhs;
    k_permute_in<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b, ld, N, nrhs, perm, out);
    count_launches(1);
}

template <typename T>
__global__ void k_permute_out(const T* in, int64_t N, int nrhs, const int64_t* perm, double* x, int64_t ld) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * nrhs) return;
    int64_t i = t / nrhs;
    int j = (int)(t - i * nrhs);
    x[perm[i] + (int64_t)j * ld] = (double)in[t];
}

template <typename T>
void launch_permute_out(const T* in, int64_t N, int nrhs, const int64_t* perm, double* x, int64_t ld,
                        cudaStream_t st) {
    int64_t tot = N * nrhs;
    k_permute_out<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, N, nrhs, perm, x, ld);
    count_launches(1);
}

#define IFMM_INSTANTIATE(T)                                                                                     \
    template void launch_factor_colour<T>(const LevelView<T>&, const int*, int, int, int, int, cudaStream_t,    \
                                          cudaEvent_t*, const int2*, const LevelView<T>*);                      \
    template void launch_forward_colour<T>(const LevelView<T>&, const int*, int, int, const int64_t*, T*, T*,   \
                                           T*, int, cudaStream_t);                                              \
    template void launch_backward_colour<T>(const LevelView<T>&, const int*, int, int, const int64_t*,          \
                                            const T*, T*, const T*, T*, int, T*, int64_t, int*, int,            \
                                            cudaStream_t);                                                      \
    template void launch_init_level<T>(const LevelView<T>&, int, const double*, const int64_t*, const double*, \
                                       const int64_t*, int, const int*, const double*, const int*, const int*, \
                                       const LevelView<T>*, cudaStream_t);                                      \
    template void launch_root_gather<T>(const LevelView<T>&, const int64_t*, double*, int, cudaStream_t);      \
    template void launch_level_scale<T>(const LevelView<T>&, double*, cudaStream_t);                            \
    template void launch_root_apply<T>(const double*, int, const T*, T*, int, cudaStream_t);                  \
    template void launch_permute_in<T>(const double*, int64_t, int64_t, int, const int64_t*, T*, cudaStream_t); \
    template void launch_permute_out<T>(const T*, int64_t, int, const int64_t*, double*, int64_t, cudaStream_t);

IFMM_INSTANTIATE(double)
IFMM_INSTANTIATE(float)

// the replay (Algorithm 2) also runs on double-float copies of FP64 factors
template void launch_forward_colour<dfl>(const LevelView<dfl>&, const int*, int, int, const int64_t*, dfl*, dfl*,
                                         dfl*, int, cudaStream_t);
template void launch_backward_colour<dfl>(const LevelView<dfl>&, const int*, int, int, const int64_t*, const dfl*,
                                          dfl*, const dfl*, dfl*, int, dfl*, int64_t, int*, int, cudaStream_t);
template void launch_root_apply<dfl>(const double*, int, const dfl*, dfl*, int, cudaStream_t);
template void launch_permute_in<dfl>(const double*, int64_t, int64_t, int, const int64_t*, dfl*, cudaStream_t);
template void launch_permute_out<dfl>(const dfl*, int64_t, int, const int64_t*, double*, int64_t, cudaStream_t);

}  // namespace ifmm
