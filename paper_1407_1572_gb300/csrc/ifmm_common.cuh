// ifmm_common.cuh -- device helpers shared by the CUDA kernels of the IFMM library (sm_103a).
//
// CTA-wide reductions, a tiled CTA GEMM with functor loaders and epilogue, in-place
// Gauss-Jordan inversion with partial pivoting, and Householder QR with column pivoting.
// Everything here runs inside one thread block; the callers give each block one box.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <type_traits>

#include "ifmm_internal.h"

#define IFMM_DEVINL __device__ __forceinline__

namespace ifmm {

constexpr int kThreads = 256;  // block size of every per-box kernel

IFMM_DEVINL int colour_of(int ix, int iy) { return (ix % 3) + 3 * (iy % 3); }

template <typename T>
IFMM_DEVINL T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block; `red` holds >= 32 entries of shared scratch
template <typename T>
__device__ T block_sum(T v, T* red) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
    return s;
}

template <typename T>
__device__ T block_max(T v, T* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = red[0];
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 1; i < nw; ++i) s = fmax(s, red[i]);
    return s;
}

// argmax of v over the block with ties to the lowest index; returns the index (or -1 when every
// thread passed idx < 0). vred/ired: >= 32 entries of shared scratch each.
__device__ inline int block_argmax(double v, int idx, double* vred, int* ired, double* vout) {
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (oi >= 0 && (idx < 0 || ov > v || (ov == v && oi < idx))) { v = ov; idx = oi; }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { vred[w] = v; ired[w] = idx; }
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    double bv = vred[0];
    int bi = ired[0];
    for (int i = 1; i < nw; ++i) {
        int oi = ired[i];
        double ov = vred[i];
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
    }
    if (vout) *vout = bv;
    return bi;
}

// ---------------------------------------------------------------------------------------------
// CTA GEMM: for (i, j) in [0, M) x [0, N): epi(i, j, sum_k la(i, k) * lb(k, j)).
// Output tiles of 64 x 64; the tiles with index = tile0 (mod tstride) belong to this block (one
// pair block can be spread over several blocks). `smem` holds gemm_smem<Acc>::value elements.
//  - FP32: register-tiled, 4 x 4 outputs per thread, k-steps of 16 (shared-memory bandwidth is
//    the limit at the FP32 rate).
//  - FP64: exact extent — each thread owns the outputs tid + 256 u of the tile that exist, so no
//    padded multiply-adds reach the FP64 pipe (the limit at the FP64 rate); k-steps of 32.
// ---------------------------------------------------------------------------------------------
template <typename Acc> struct gemm_smem { static constexpr int value = 2 * 16 * 65; };
template <> struct gemm_smem<double> { static constexpr int value = 2 * 32 * 64; };
template <> struct gemm_smem<dfl> { static constexpr int value = 2 * 32 * 33; };

// ---------------------------------------------------------------------------------------------
// double-float arithmetic (the type is declared in ifmm_internal.h). The intrinsics keep the
// compiler from contracting the error-free transformations.
// ---------------------------------------------------------------------------------------------
// s += a * b: the exact product a.hi b.hi = p + e (FMA), the cross terms a.hi b.lo + a.lo b.hi added
// to e (a.lo b.lo dropped), p added to s.hi exactly (TwoSum), the rounding errors gathered in s.lo
IFMM_DEVINL void dfl_fma_acc(dfl& s, dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float t = __fadd_rn(s.hi, p);
    const float z = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}
// renormalise: hi = fl(hi + lo), lo = the exact remainder (TwoSum)
IFMM_DEVINL dfl dfl_norm(dfl a) {
    const float t = __fadd_rn(a.hi, a.lo);
    const float z = __fsub_rn(t, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, z)), __fsub_rn(a.lo, z));
    return dfl(t, err);
}
IFMM_DEVINL dfl operator+(dfl a, dfl b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float z = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return dfl_norm(dfl(s, e));
}
IFMM_DEVINL dfl operator-(dfl a, dfl b) { return a + dfl(-b.hi, -b.lo); }
// scalar helpers of the pivot elimination (FP64): magnitude for the pivot search, product, s - f p
IFMM_DEVINL double sc_mag(double v) { return fabs(v); }
IFMM_DEVINL double sc_mul(double a, double b) { return a * b; }
IFMM_DEVINL double sc_fms(double s, double f, double p) { return s - f * p; }
IFMM_DEVINL double sc_neg(double v) { return -v; }
IFMM_DEVINL dfl& operator+=(dfl& a, dfl b) {
    a = a + b;
    return a;
}

// CTA GEMM in double-float: output tiles of 32 x 32, each of the 256 threads owns 2 x 2 outputs
// (rows ty, ty + 16, columns tx, tx + 16), k-steps of 32 staged in padded shared tiles; the next
// k-step's operands (4 of A and 4 of B per thread) are loaded into registers while the current one
// is multiplied. About 11 FP32 operations per multiply-add and 4 shared loads per 4 multiply-adds:
// FP32-pipe bound.
template <class LA, class LB, class EPI>
__device__ void cta_gemm_dfl(int M, int N, int K, LA la, LB lb, EPI epi, dfl* smem, int tile0, int tstride) {
    constexpr int TM = 32, TN = 32, KC = 32, LDA = TM + 1, LDB = TN + 1;
    dfl* As = smem;              // [KC][LDA] : As[k][i]
    dfl* Bs = smem + KC * LDA;   // [KC][LDB] : Bs[k][j]
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int tn = (N + TN - 1) / TN, tm = (M + TM - 1) / TM;
    // staging: element u of this thread is tid + 256 u (u < 4) of the 32 x 32 chunk; A as (i, k) =
    // (t / KC, t % KC), B as (k, j) = (t / TN, t % TN)
    for (int tile = tile0; tile < tm * tn; tile += tstride) {
        const int m0 = (tile / tn) * TM, n0 = (tile % tn) * TN;
        dfl acc[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) acc[a][b] = dfl(0.0f, 0.0f);
        // operands that are double-float already (the replay, the matvec) are prefetched into
        // registers one k-step ahead; FP64 operands (split while staged) are staged directly,
        // where the extra registers would cost more occupancy than the overlap gains
        constexpr bool kPrefetch = std::is_same<std::decay_t<decltype(la(0, 0))>, dfl>::value &&
                                   std::is_same<std::decay_t<decltype(lb(0, 0))>, dfl>::value;
        if constexpr (!kPrefetch) {
            for (int k0 = 0; k0 < K; k0 += KC) {
                for (int t = tid; t < TM * KC; t += 256) {
                    const int i = t / KC, k = t - i * KC;
                    const int gi = m0 + i, gk = k0 + k;
                    As[k * LDA + i] = (gi < M && gk < K) ? dfl(la(gi, gk)) : dfl(0.0f, 0.0f);
                }
                for (int t = tid; t < KC * TN; t += 256) {
                    const int k = t / TN, j = t - k * TN;
                    const int gk = k0 + k, gj = n0 + j;
                    Bs[k * LDB + j] = (gk < K && gj < N) ? dfl(lb(gk, gj)) : dfl(0.0f, 0.0f);
                }
                __syncthreads();
                const int kc = min(KC, K - k0);
                for (int kk = 0; kk < kc; ++kk) {
                    const dfl a0 = As[kk * LDA + ty], a1 = As[kk * LDA + ty + 16];
                    const dfl b0 = Bs[kk * LDB + tx], b1 = Bs[kk * LDB + tx + 16];
                    dfl_fma_acc(acc[0][0], a0, b0);
                    dfl_fma_acc(acc[0][1], a0, b1);
                    dfl_fma_acc(acc[1][0], a1, b0);
                    dfl_fma_acc(acc[1][1], a1, b1);
                }
                __syncthreads();
            }
        } else {
        dfl ra[4], rb[4];
        auto fetch = [&](int k0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = tid + 256 * u;
                const int i = t / KC, k = t - i * KC;
                const int gi = m0 + i, gk = k0 + k;
                ra[u] = (gi < M && gk < K) ? dfl(la(gi, gk)) : dfl(0.0f, 0.0f);
                const int kb = t / TN, jb = t - kb * TN;
                const int gkb = k0 + kb, gj = n0 + jb;
                rb[u] = (gkb < K && gj < N) ? dfl(lb(gkb, gj)) : dfl(0.0f, 0.0f);
            }
        };
        if (K > 0) fetch(0);
        for (int k0 = 0; k0 < K; k0 += KC) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = tid + 256 * u;
                const int i = t / KC, k = t - i * KC;
                As[k * LDA + i] = ra[u];
                const int kb = t / TN, jb = t - kb * TN;
                Bs[kb * LDB + jb] = rb[u];
            }
            __syncthreads();
            if (k0 + KC < K) fetch(k0 + KC);
            const int kc = min(KC, K - k0);
            for (int kk = 0; kk < kc; ++kk) {
                const dfl a0 = As[kk * LDA + ty], a1 = As[kk * LDA + ty + 16];
                const dfl b0 = Bs[kk * LDB + tx], b1 = Bs[kk * LDB + tx + 16];
                dfl_fma_acc(acc[0][0], a0, b0);
                dfl_fma_acc(acc[0][1], a0, b1);
                dfl_fma_acc(acc[1][0], a1, b0);
                dfl_fma_acc(acc[1][1], a1, b1);
            }
            __syncthreads();
        }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int gi = m0 + ty + 16 * a, gj = n0 + tx + 16 * b;
                if (gi < M && gj < N) epi(gi, gj, dfl_norm(acc[a][b]));
            }
    }
}

template <typename Acc, class LA, class LB, class EPI>
__device__ void cta_gemm_exact(int M, int N, int K, LA la, LB lb, EPI epi, Acc* smem, int tile0, int tstride) {
    constexpr int TM = 64, TN = 64, KC = 32, PER = 16;
    Acc* As = smem;             // [KC][TM] : As[k][i]
    Acc* Bs = smem + KC * TM;   // [KC][TN] : Bs[k][j]
    const int tid = threadIdx.x;
    const int tn = (N + TN - 1) / TN, tm = (M + TM - 1) / TM;
    for (int tile = tile0; tile < tm * tn; tile += tstride) {
        const int m0 = (tile / tn) * TM, n0 = (tile % tn) * TN;
        const int mm = min(TM, M - m0), nn = min(TN, N - n0), tot = mm * nn;
        const int cnt = tot > tid ? (tot - tid + 255) / 256 : 0;
        int oi[PER], oj[PER];
        Acc acc[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            int o = tid + 256 * u;
            oi[u] = o / nn;
            oj[u] = o - oi[u] * nn;
            acc[u] = Acc(0);
        }
        for (int k0 = 0; k0 < K; k0 += KC) {
            const int kc = min(KC, K - k0);
            for (int t = tid; t < mm * KC; t += 256) {
                int i = t / KC, k = t - i * KC;
                As[k * TM + i] = k < kc ? Acc(la(m0 + i, k0 + k)) : Acc(0);
            }
            for (int t = tid; t < KC * nn; t += 256) {
                int k = t / nn, j = t - k * nn;
                Bs[k * TN + j] = k < kc ? Acc(lb(k0 + k, n0 + j)) : Acc(0);
            }
            __syncthreads();
            for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
                for (int u = 0; u < PER; ++u)
                    if (u < cnt) acc[u] = fma(As[kk * TM + oi[u]], Bs[kk * TN + oj[u]], acc[u]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < PER; ++u)
            if (u < cnt) epi(m0 + oi[u], n0 + oj[u], acc[u]);
    }
}

template <typename Acc, class LA, class LB, class EPI>
__device__ void cta_gemm(int M, int N, int K, LA la, LB lb, EPI epi, Acc* smem, int tile0 = 0, int tstride = 1) {
    if constexpr (std::is_same<Acc, dfl>::value) {
        cta_gemm_dfl(M, N, K, la, lb, epi, smem, tile0, tstride);
        return;
    } else if constexpr (sizeof(Acc) == 8) {
        cta_gemm_exact<Acc>(M, N, K, la, lb, epi, smem, tile0, tstride);
        return;
    } else {
        constexpr int BM = 64, BN = 64, BK = 16, LDS = 65;
        Acc* As = smem;             // [BK][LDS] : As[k][i]
        Acc* Bs = smem + BK * LDS;  // [BK][LDS] : Bs[k][j]
        const int tid = threadIdx.x;
        const int tx = tid & 15, ty = tid >> 4;
        const int tn = (N + BN - 1) / BN, tm = (M + BM - 1) / BM;
        for (int tile = tile0; tile < tm * tn; tile += tstride) {
            const int m0 = (tile / tn) * BM, n0 = (tile % tn) * BN;
            Acc acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = Acc(0);
            for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int ii = (tid >> 4) + 16 * q, kk = tid & 15;
                    int gi = m0 + ii, gk = k0 + kk;
                    As[kk * LDS + ii] = (gi < M && gk < K) ? Acc(la(gi, gk)) : Acc(0);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int kk = (tid >> 6) + 4 * q, jj = tid & 63;
                    int gk = k0 + kk, gj = n0 + jj;
                    Bs[kk * LDS + jj] = (gk < K && gj < N) ? Acc(lb(gk, gj)) : Acc(0);
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    Acc av[4], bv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) av[a] = As[kk * LDS + ty + 16 * a];
#pragma unroll
                    for (int b = 0; b < 4; ++b) bv[b] = Bs[kk * LDS + tx + 16 * b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    int gi = m0 + ty + 16 * a, gj = n0 + tx + 16 * b;
                    if (gi < M && gj < N) epi(gi, gj, acc[a][b]);
                }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// In-place inversion of the s x s matrix A (leading dimension lda, FP64) by Gauss-Jordan
// elimination with partial pivoting (ties to the lowest row). perm: s ints of scratch, col: s
// doubles of scratch (shared or global). Returns false if a pivot column is exactly zero.
// ---------------------------------------------------------------------------------------------
__device__ inline bool cta_gauss_jordan(double* A, int s, int lda, int* perm, double* col, double* vred,
                                        int* ired) {
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ double s_piv;
    __shared__ int s_ok;
    for (int k = 0; k < s; ++k) {
        double best = -1.0;
        int bi = -1;
        for (int i = k + tid; i < s; i += nt) {
            double v = fabs(A[(size_t)i * lda + k]);
            if (bi < 0 || v > best) { best = v; bi = i; }
        }
        double bv;
        int p = block_argmax(best, bi, vred, ired, &bv);
        if (tid == 0) {
            perm[k] = p;
            s_ok = (p >= 0 && bv > 0.0 && isfinite(bv)) ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) return false;
        if (p != k)
            for (int j = tid; j < s; j += nt) {
                double t = A[(size_t)k * lda + j];
                A[(size_t)k * lda + j] = A[(size_t)p * lda + j];
                A[(size_t)p * lda + j] = t;
            }
        __syncthreads();
        if (tid == 0) s_piv = A[(size_t)k * lda + k];
        __syncthreads();
        double d = 1.0 / s_piv;
        for (int j = tid; j < s; j += nt) {
            if (j == k) A[(size_t)k * lda + k] = d;
            else A[(size_t)k * lda + j] *= d;
        }
        for (int i = tid; i < s; i += nt) col[i] = A[(size_t)i * lda + k];
        __syncthreads();
        // rows i != k: A[i][j] -= col[i] * A[k][j] (j != k); A[i][k] = -col[i] * d. Element
        // t = i s + j walked in steps of nt = dr s + dc (no division per element).
        {
            const int dr = nt / s, dc = nt - dr * s;
            for (int i = tid / s, j = tid - (tid / s) * s; i < s;) {
                if (i != k) {
                    if (j == k) A[(size_t)i * lda + k] = -col[i] * d;
                    else A[(size_t)i * lda + j] -= col[i] * A[(size_t)k * lda + j];
                }
                i += dr;
                j += dc;
                if (j >= s) { j -= s; ++i; }
            }
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int k = s - 1; k >= 0; --k) {
        int p = perm[k];
        if (p != k)
            for (int i = tid; i < s; i += nt) {
                double t = A[(size_t)i * lda + k];
                A[(size_t)i * lda + k] = A[(size_t)i * lda + p];
                A[(size_t)i * lda + p] = t;
            }
        __syncthreads();
    }
    return true;
}

// ---------------------------------------------------------------------------------------------
// Householder QR with column pivoting of the m x nc matrix A (FP64, leading dimension lda,
// overwritten). Columns are taken while the largest remaining column norm exceeds
// tol * (largest column norm of A); ties go to the lowest column. On return Q (m x rank, ldq)
// holds orthonormal columns, Rt (rank x nc, ldr) with A = Q Rt, and the rank is returned.
// Scratch: vbuf (m doubles per reflector, rank reflectors: m * min(m, nc)), beta (nc), cperm (nc),
// red (>= 32 doubles), ired (>= 32 ints).
// ---------------------------------------------------------------------------------------------
__device__ inline int cta_cpqr(double* A, int m, int nc, int lda, double tol, double* Q, int ldq,
                               double* Rt, int ldr, double* vbuf, double* beta, int* cperm, double* red,
                               int* ired) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    __shared__ double s_first, s_alpha, s_beta;
    __shared__ int s_rank;
    for (int j = tid; j < nc; j += nt) cperm[j] = j;
    if (tid == 0) { s_first = -1.0; s_rank = 0; }
    __syncthreads();
    int kmax = m < nc ? m : nc;
    int rank = 0;
    for (int k = 0; k < kmax; ++k) {
        // norms of the remaining columns, one warp per column
        double best = -1.0;
        int bi = -1;
        for (int j = k + warp; j < nc; j += nw) {
            double s = 0.0;
            for (int i = k + lane; i < m; i += 32) s += A[(size_t)i * lda + j] * A[(size_t)i * lda + j];
            s = warp_sum(s);
            double v = sqrt(s);
            if (bi < 0 || v > best) { best = v; bi = j; }
        }
        if (lane != 0) bi = -1;
        double bv;
        int jb = block_argmax(best, bi, red, ired, &bv);
        if (tid == 0 && s_first < 0.0) s_first = bv;
        __syncthreads();
        if (!(bv > tol * s_first) || bv == 0.0) break;
        if (jb != k) {
            for (int i = tid; i < m; i += nt) {
                double t = A[(size_t)i * lda + k];
                A[(size_t)i * lda + k] = A[(size_t)i * lda + jb];
                A[(size_t)i * lda + jb] = t;
            }
            if (tid == 0) { int t = cperm[k]; cperm[k] = cperm[jb]; cperm[jb] = t; }
        }
        __syncthreads();
        double* v = vbuf + (size_t)k * m;
        for (int i = tid; i < m; i += nt) v[i] = (i >= k) ? A[(size_t)i * lda + k] : 0.0;
        __syncthreads();
        if (tid == 0) {
            double alpha = v[k] >= 0.0 ? -bv : bv;
            v[k] -= alpha;
            s_alpha = alpha;
        }
        __syncthreads();
        double vtv = 0.0;
        for (int i = k + tid; i < m; i += nt) vtv += v[i] * v[i];
        vtv = block_sum(vtv, red);
        if (tid == 0) { s_beta = vtv > 0.0 ? 2.0 / vtv : 0.0; beta[k] = s_beta; }
        __syncthreads();
        double bt = s_beta;
        // apply H = I - beta v v^T to columns k..nc-1, one warp per column
        for (int j = k + warp; j < nc; j += nw) {
            double s = 0.0;
            for (int i = k + lane; i < m; i += 32) s += v[i] * A[(size_t)i * lda + j];
            s = warp_sum(s) * bt;
            for (int i = k + lane; i < m; i += 32) A[(size_t)i * lda + j] -= s * v[i];
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < m; i += nt) A[(size_t)i * lda + k] = 0.0;
        if (tid == 0) A[(size_t)k * lda + k] = s_alpha;
        ++rank;
        __syncthreads();
    }
    // Q = H_0 ... H_{rank-1} [I; 0]
    for (int t = tid; t < m * rank; t += nt) {
        int i = t / rank, j = t - i * rank;
        Q[(size_t)i * ldq + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = rank - 1; k >= 0; --k) {
        const double* v = vbuf + (size_t)k * m;
        double bt = beta[k];
        for (int j = warp; j < rank; j += nw) {
            double s = 0.0;
            for (int i = k + lane; i < m; i += 32) s += v[i] * Q[(size_t)i * ldq + j];
            s = warp_sum(s) * bt;
            for (int i = k + lane; i < m; i += 32) Q[(size_t)i * ldq + j] -= s * v[i];
        }
        __syncthreads();
    }
    // Rt[:, cperm[j]] = R[0:rank, j]
    for (int t = tid; t < rank * nc; t += nt) {
        int i = t / nc, j = t - i * nc;
        Rt[(size_t)i * ldr + cperm[j]] = A[(size_t)i * lda + j];
    }
    __syncthreads();
    return rank;
}

}  // namespace ifmm
