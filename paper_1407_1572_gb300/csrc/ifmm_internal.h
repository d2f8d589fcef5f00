// ifmm_internal.h -- structures shared by the host orchestration and the CUDA kernels.
#pragma once
#include <cstdint>
#include <map>
#include <tuple>
#include <cuda_runtime.h>

namespace ifmm {

// Double-float number hi + lo (two FP32 values, |lo| <= ulp(hi) / 2 when normalised): about 48
// significand bits with FP32's exponent range. GB300 runs FP32 at 64 times its FP64 rate, so the
// replay and the FMM matvec of the mixed-precision solve keep their operands in this form and run
// on the FP32 pipe (multiply-adds by the exact-product and exact-sum transformations of Dekker and
// Knuth); FP64 values split as hi = fl32(d), lo = fl32(d - hi).
struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // On the device the split works on the bit pattern (integer and FP32 operations only; the FP64
    // pipe is 64 times slower): hi = d truncated to 24 significant bits, lo = the remaining 29
    // bits rounded to 24, both exact scalings of the double's fields. Exponents whose hi or lo
    // would leave the FP32 normal range take the FP64 formula.
    __host__ __device__ explicit dfl(double d) {
#ifdef __CUDA_ARCH__
        const unsigned long long b = (unsigned long long)__double_as_longlong(d);
        const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
        if (e >= 949u && e <= 1150u) {
            const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
            hi = __uint_as_float(sgn | ((e - 896u) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu));
            const float scale = __uint_as_float((e - 948u) << 23);  // 2^(e - 1075)
            const float m = __uint2float_rn((unsigned)b & 0x1FFFFFFFu);
            lo = __uint_as_float(__float_as_uint(__fmul_rn(m, scale)) | sgn);
            return;
        }
#endif
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
    __host__ __device__ explicit dfl(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// kernels launched by this library in this process (every launcher adds its launches)
void count_launches(int n);
long long launches_so_far();
// entries of the factorisation's device counter array (LevelView::counters)
constexpr int kCounters = 16;
// largest cluster one compression launch may use (1, 2, 4, 8 or 16); -1 for any other value
int set_compress_cluster(int c);

// device status flags (bit set by any block that fails)
enum : int { DEV_ERR_SINGULAR = 1, DEV_ERR_OVERFLOW = 2, DEV_ERR_RANGE = 4, DEV_ERR_SIZE = 8, DEV_ERR_TIMEOUT = 16 };

// Digit slabs of the stored factors for the tensor-core replay (ifmm_tc.cuh: operands split once,
// multiplied by every replay), twelve operands per box e: 0 = Pi_e with rows s, K = n (forward
// replay), 1 = Pi_e with rows n, K = s (back substitution), 2 + d = the C panel of neighbour
// direction d (rows w_q, K = n), 11 = the B panels of all directions side by side (rows n, K = the
// sum of the widths). slab == nullptr: no slabs (the replay splits nothing and multiplies as before).
constexpr int kSlabRecs = 12;
struct SlabSet {
    const uint8_t* slab;
    const int* rexp;
    const int64_t* soff;   // [nb * kSlabRecs] byte offset of the operand's slab (-1: none)
    const int64_t* eoff;   // [nb * kSlabRecs] offset of its row exponents
};

// Geometry of one level of the uniform tree (Section 4.2), in d = 2 (quadtree) or d = 3 (octree,
// the paper's extension to three dimensions). Box b sits at grid cell (b mod s, (b / s) mod s,
// b / s^2) (z = 0 in 2D). Its neighbour in direction dq (0 <= dq < 3^d) is the cell displaced by
// (dq mod 3 - 1, (dq / 3) mod 3 - 1, dq / 9 - 1); direction 3^d / 2 (4 or 13) is the box itself,
// and a lower direction index means a lower grid index. The 6^d region of a box p is made of the
// children of its parent's neighbours: every neighbour and every interaction-list box of p is in it.
// Colour (reading R1): (x mod 3) + 3 (y mod 3) + 9 (z mod 3), 3^d colours.
struct Cell { int x, y, z; };
#if defined(__CUDACC__)
#define IFMM_HD __host__ __device__ __forceinline__
#else
#define IFMM_HD inline
#endif
IFMM_HD Cell cell_of(int b, int side, int dim) {
    return Cell{b % side, (b / side) % side, dim == 3 ? b / (side * side) : 0};
}
IFMM_HD int cell_index(Cell c, int side) { return c.x + side * (c.y + side * c.z); }
IFMM_HD bool cell_in(Cell c, int side) {
    return c.x >= 0 && c.y >= 0 && c.z >= 0 && c.x < side && c.y < side && c.z < side;
}
IFMM_HD Cell cell_dir(Cell c, int dq, int dim) {
    return Cell{c.x + dq % 3 - 1, c.y + (dq / 3) % 3 - 1, dim == 3 ? c.z + dq / 9 - 1 : c.z};
}
IFMM_HD int dir_index(Cell from, Cell to, int dim) {
    return (to.x - from.x + 1) + 3 * (to.y - from.y + 1) + (dim == 3 ? 9 * (to.z - from.z + 1) : 0);
}
IFMM_HD int cheb_dist(Cell a, Cell b) {
    const int dx = a.x > b.x ? a.x - b.x : b.x - a.x, dy = a.y > b.y ? a.y - b.y : b.y - a.y;
    const int dz = a.z > b.z ? a.z - b.z : b.z - a.z;
    return dx > dy ? (dx > dz ? dx : dz) : (dy > dz ? dy : dz);
}
IFMM_HD int cell_colour(Cell c) { return (c.x % 3) + 3 * (c.y % 3) + 9 * (c.z % 3); }
IFMM_HD int region_index(Cell p, Cell q, int dim) {
    return (q.x - 2 * (p.x >> 1) + 2) + 6 * (q.y - 2 * (p.y >> 1) + 2) + (dim == 3 ? 36 * (q.z - 2 * (p.z >> 1) + 2) : 0);
}
IFMM_HD Cell region_cell(Cell p, int j, int dim) {
    return Cell{2 * (p.x >> 1) - 2 + j % 6, 2 * (p.y >> 1) - 2 + (j / 6) % 6, dim == 3 ? 2 * (p.z >> 1) - 2 + j / 36 : p.z};
}
IFMM_HD int ndirs(int dim) { return dim == 3 ? 27 : 9; }
IFMM_HD int nregion(int dim) { return dim == 3 ? 216 : 36; }
IFMM_HD int ncolours(int dim) { return dim == 3 ? 27 : 9; }
// child c = a + 2 b (+ 4 e) of a box: cell (2 x + a, 2 y + b, 2 z + e)
IFMM_HD Cell child_cell(Cell c, int ch) { return Cell{2 * c.x + (ch & 1), 2 * c.y + ((ch >> 1) & 1), 2 * c.z + ((ch >> 2) & 1)}; }

// Device view of one tree level during elimination (Algorithm 1) and replay (Algorithm 2).
// Box b of level k sits at grid position (b % side, b / side). Its particle unknowns x_b number
// n[b]; its multipoles y_b and locals z_b number r[b] (the rank, grows by compression).
//
// blk: for every box p and every box q of p's 6^d region (region_index), the block between the
// active equation of p and the active unknown of q (Algorithm 1's P2P, P2L, M2P or M2L by
// elimination status) for neighbours, the M2L block for interaction-list boxes. Offsets
// boff[p * nreg + j] (-1: no block), leading dimension bld.
template <typename T>
struct LevelView {
    int k, side, nb, RC;       // level, boxes per side, boxes, rank cap of the level
    int dim, nd, ctr, nreg;    // dimension, 3^d directions, the box's own direction, 6^d region
    int nmax;                  // largest n at the level (sizes the tile split of big blocks)
    const int* n;              // [nb] particle count (leaf) or sum of the children's ranks
    int* r;                    // [nb] rank
    const int64_t* voff;       // [nb+1] prefix of n: rows of box b in level vectors and in W
    const int64_t* boff;       // [nb * nreg]
    const int* bld;            // [nb * nreg]
    T* blk;
    T* W;                      // (sum n) x RC: L2P_bb = W rows voff[b].., P2M_bb = its transpose
    // factors kept for the solve
    const int64_t* pioff;      // [nb] inverse pivot block, s x s with leading dimension pild
    const int* pild;
    T* Pi;
    const int64_t* cpoff;      // [nb * nd] C panel of neighbour direction d: rows of the neighbour
    T* Cp;                     //        at column x_b (w x n_b, leading dimension n_b)
    const int64_t* bpoff;      // [nb * nd] B panel: row P2P_b at the neighbour's column (n_b x w,
    T* Bp;                     //        leading dimension w)
    // per-colour scratch (offsets restart at every colour)
    const int64_t* xsoff;      // [nb] X = Pi [B; 0] for every column block, s x xsld
    const int* xsld;
    T* Xs;
    const int64_t* fsoff;      // [nb * nd * nd] well-separated fill of ordered pair (dp, dq)
    T* Fs;
    T* Fs2;                    // same layout: intermediate of the redirect
    const int64_t* rsoff;      // [nb * nd] residual of the fill being compressed
    T* Rs;
    const int64_t* cwsoff;     // [nb * nd] the compression's FP64 work arrays (basis vector, coefficients,
    double* Cws;               //        column norms) when they do not fit in shared memory
    double* pws;               // FP64 pivot workspace for blocks too large for shared memory
    const int64_t* psoff;      // [nb]
    int* status;               // device error bits (DEV_ERR_*)
    double* counters;          // [0] schur flops, [1] schur bytes, [2] all factor flops,
                               // [3] pivot, [4] panel, [5] compress, [6] redirect flops,
                               // [7] the projection part of [5], [8] its re-orthogonalisation
                               // part (kCounters entries)
    double eps, sA;
    int tau_ref;
    int symmetric;             // kernel symmetric: F_pq = F_qp^T in exact arithmetic
    int gemm_dfl;              // FP64 level data, panel and Schur products in double-float (FP32 pipe)
    int gemm_tc;               // with gemm_dfl: the Schur products on the tensor cores (ifmm_tc.cuh)
    SlabSet sl;                // digit slabs of the factors for the tensor-core replay
};

// The boxes one launch of a factor kernel eliminates: the boxes of one colour of one level of one
// system (`boxes`, the level view passed to the kernel by value), or the work items of a batch of
// systems eliminated together (items[i] = (index of the system's level view in `views`, box)).
template <typename T>
struct BoxList {
    const int* boxes;
    const int2* items;
    const LevelView<T>* views;
#ifdef __CUDACC__
    __device__ __forceinline__ const LevelView<T>& view(const LevelView<T>& L0, int i) const {
        return items ? views[items[i].x] : L0;
    }
    __device__ __forceinline__ int box(int i) const { return items ? items[i].y : boxes[i]; }
#endif
};

// Level vectors of the replay: for box b of level k, rows voff[b].. of the level-k vector hold
// its particle rows; rows yoff[b].. of the level-(k-1) vector (the root vector at k = 2) hold its
// multipole / local rows.
struct SolveView {
    const int64_t* yoff;
    int nrhs;
};

// ---- launchers (ifmm_factor.cu) -----------------------------------------------------------
// autotuner of the panel / Schur launch splits: candidate forcing, event records, the table
void tune_set_force(int panel, int schur);
void tune_record(bool on);
std::map<std::tuple<int, int, int, int>, double> tune_collect(int kernel);
void tune_table_set(const std::map<std::tuple<int, int, int, int>, int>& t);
std::map<std::tuple<int, int, int, int>, int> tune_table_get();
// ev (optional): 6 events recorded before each of the five launches and after the last
template <typename T>
// smem_pivot_s: the level's bound on a pivot's size; exact_sizing: read the colour's actual largest
// pivot back (a stream synchronisation) to size the pivot launch
// items / views (nullptr for one system): the blocks of a batch of systems (BoxList)
void launch_factor_colour(const LevelView<T>& L, const int* boxes, int nboxes, int colour, int smem_pivot_s,
                          int exact_sizing, cudaStream_t st, cudaEvent_t* ev, const int2* items = nullptr,
                          const LevelView<T>* views = nullptr);
template <typename T>
void launch_forward_colour(const LevelView<T>& L, const int* boxes, int nboxes, int colour, const int64_t* yoff,
                           T* vec_k, T* vec_km1, T* vx, int nrhs, cudaStream_t st);
// part (part_cap elements) and cnt (cnt_cap ints, zero on entry and on return): split-K scratch
// for colours with few boxes; NULL disables the split
template <typename T>
void launch_backward_colour(const LevelView<T>& L, const int* boxes, int nboxes, int colour, const int64_t* yoff,
                            const T* rhs_k, T* x_k, const T* x_km1, T* wtmp, int nrhs, T* part, int64_t part_cap,
                            int* cnt, int cnt_cap, cudaStream_t st);
template <typename T>
void launch_init_level(const LevelView<T>& L, int is_leaf, const double* p2p0, const int64_t* p2p0_off,
                       const double* W0, const int64_t* w0_rowoff, int r0, const int* xoffs,
                       const double* far0, const int* rank0, const int* rank0_child, const LevelView<T>* child,
                       cudaStream_t st);
template <typename T>
void launch_level_scale(const LevelView<T>& L, double* out, cudaStream_t st);
// split the stored factors of the boxes of one colour into digit slabs (L.sl, written)
void launch_presplit(const LevelView<double>& L, uint8_t* slab, int* rexp, const int* boxes, int nboxes, int colour,
                     cudaStream_t st);
template <typename T>
void launch_root_gather(const LevelView<T>& L2, const int64_t* rootoff, double* D, int M, cudaStream_t st);
void launch_dense_invert(double* D, int M, int* perm, double* col, int* status, cudaStream_t st);
template <typename T>
void launch_root_apply(const double* Dinv, int M, const T* rhs, T* x, int nrhs, cudaStream_t st);
template <typename T>
void launch_permute_in(const double* b, int64_t ld, int64_t N, int nrhs, const int64_t* perm, T* out,
                       cudaStream_t st);
template <typename T>
void launch_permute_out(const T* in, int64_t N, int nrhs, const int64_t* perm, double* x, int64_t ld,
                        cudaStream_t st);

// ---- build and matvec (ifmm_build.cu) -----------------------------------------------------
struct BuildArgs {
    int64_t N;
    int depth, p, r0, kernel;
    double kparam0, diag, x0, y0, L;
    int dim;       // 2 or 3
    double z0;     // 3D: lower z of the root cube
};
void launch_leaf_keys(const double* pts, int64_t N, int depth, int dim, double x0, double y0, double z0, double L,
                      unsigned long long* keys, int64_t npad, int* status, cudaStream_t st);
void launch_bitonic_sort(unsigned long long* keys, int64_t npad, cudaStream_t st);
void launch_scatter_sorted(const unsigned long long* keys, const double* pts, int64_t N, int dim, int64_t* perm,
                           double* px, double* py, double* pz, int* leaf_count, int depth, cudaStream_t st);
void launch_leaf_basis(const BuildArgs& a, const double* px, const double* py, const double* pz,
                       const int64_t* leaf_start, const int* leaf_count, const double* cheb, double* W0, double* Rt,
                       int* rank0, int max_n, const double* U, const int* rsvd, cudaStream_t st);
void launch_svd_level(const BuildArgs& a, int k, double svd_eps, const double* cheb, const double* Tc,
                      const double* Up, const double* sp, const int* rp, double* U, double* sig, int* rk,
                      double* scratch, cudaStream_t st);
size_t svd_scratch_doubles(int r0, int dim);
void launch_parent_basis(const BuildArgs& a, int k, const double* Rt_child, const int* rank_child,
                         const double* Tc, double* W0, double* Rt, int* rank0, const double* U, const int* rsvd,
                         cudaStream_t st);
void launch_m2l_build(const BuildArgs& a, int k, const double* cheb, const double* Rt, double* far0,
                      cudaStream_t st);
void launch_p2p_build(const BuildArgs& a, const double* px, const double* py, const double* pz,
                      const int64_t* leaf_start, const int* leaf_count, const int64_t* p2p_off, double* p2p,
                      double* sA_bits, cudaStream_t st);
// FMM matvec pieces, element type T = double (residuals) or dfl (inner Krylov steps); dim = 2 or 3
template <typename T>
void launch_mv_permute_in(const double* x, int64_t ld, int64_t N, int nrhs, const int64_t* perm, T* xt,
                          cudaStream_t st);
template <typename T>
void launch_mv_leaf_up(int dim, int depth, const T* W0, const int64_t* leaf_start, const int* leaf_count, int r0,
                       const T* xt, T* y, int nrhs, cudaStream_t st);
template <typename T>
void launch_mv_up(int dim, int k, const T* W0, int r0, const T* ychild, T* y, int nrhs, cudaStream_t st);
template <typename T>
void launch_mv_m2l(int dim, int k, const T* far0, int r0, const T* y, T* z, int nrhs, cudaStream_t st);
template <typename T>
void launch_mv_down(int dim, int k, const T* W0, int r0, const T* z, T* zchild, int nrhs, cudaStream_t st);
template <typename T>
void launch_mv_leaf_down(int dim, int depth, const T* W0, const int64_t* leaf_start, const int* leaf_count, int r0,
                         const T* z, const T* xt, const int64_t* p2p_off, const T* p2p, T* out, int nrhs,
                         cudaStream_t st);
template <typename T>
void launch_mv_permute_out(const T* yt, int64_t N, int nrhs, const int64_t* perm, double* y, int64_t ld,
                           cudaStream_t st);
// b = a split into double-float pairs, n elements
void launch_split_dfl(const double* a, dfl* b, int64_t n, cudaStream_t st);
// refinement helpers; their sums over N are reduced in a fixed order through `part`, a device
// scratch of reduction_scratch_doubles(N, nrhs, cnt) doubles (cnt: the most dot products of one call)
size_t reduction_scratch_doubles(int64_t N, int nrhs, int cnt);
void launch_axpy_norms(double* x, const double* d, int64_t N, int nrhs, int64_t ld, double* nrm, double* part,
                       cudaStream_t st);
void launch_residual(const double* b, const double* ax, double* r, int64_t N, int nrhs, int64_t ld,
                     double* nrm, double* part, cudaStream_t st);

// Krylov vectors (FP64, column-major N x nrhs, basis vector i at V + i N nrhs)
void launch_krylov_dots(const double* V, int cnt, const double* w, int64_t N, int nrhs, double* out, double* part,
                        cudaStream_t st);
void launch_krylov_lincomb(const double* V, int cnt, const double* coef, double* y, int64_t ldy, int64_t N, int nrhs,
                           cudaStream_t st);
void launch_colnorm2(const double* y, int64_t ldy, int64_t N, int nrhs, double* out, double* part, cudaStream_t st);
void launch_colscale(double* y, int64_t ldy, int64_t N, int nrhs, const double* scale, cudaStream_t st);

}  // namespace ifmm
