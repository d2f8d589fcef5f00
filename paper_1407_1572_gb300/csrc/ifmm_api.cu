// ifmm_api.cu -- C ABI (include/ifmm.h) and host orchestration of the IFMM on one GB300.
//
// The host lays out every level (offset tables for the blocks, bases, panels and per-colour
// scratch), launches the kernels colour by colour on the handle's stream, and reads back only
// the box ranks at the end of each level (they size the next level) and the status bits.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <atomic>
#include <thread>
#include <tuple>
#include <type_traits>
#include <string>
#include <vector>

#include "ifmm.h"
#include "ifmm_internal.h"
#include "ifmm_tc.cuh"

using namespace ifmm;

namespace {

struct FLevel {
    int k = 0, side = 0, nb = 0, RC = 0, smax = 0, dim = 2;
    double scale = 0.0;   // threshold reference of the level (tau_ref = 1)
    std::vector<int> n, r, r0;
    std::vector<int64_t> voff, yoff;
    std::vector<int> xoffs;   // non-leaf: 2^d + 1 offsets per box of the children's rows in x_b
    std::vector<int> boxes;
    int cstart[28] = {0};     // colour c's boxes: boxes[cstart[c] .. cstart[c + 1])
    int64_t vtot = 0;
    // device
    int* d_n = nullptr;
    int* d_r = nullptr;
    int64_t* d_voff = nullptr;
    int64_t* d_yoff = nullptr;
    int64_t* d_boff = nullptr;
    int* d_bld = nullptr;
    void* d_blk = nullptr;
    void* d_W = nullptr;
    int64_t* d_pioff = nullptr;
    int* d_pild = nullptr;
    void* d_Pi = nullptr;
    int64_t* d_cpoff = nullptr;
    void* d_Cp = nullptr;
    int64_t* d_bpoff = nullptr;
    void* d_Bp = nullptr;
    int64_t* d_xsoff = nullptr;
    int* d_xsld = nullptr;
    void* d_Xs = nullptr;
    int64_t* d_fsoff = nullptr;
    void* d_Fs = nullptr;
    void* d_Fs2 = nullptr;
    int64_t* d_rsoff = nullptr;
    void* d_Rs = nullptr;
    int64_t* d_cwsoff = nullptr;
    double* d_Cws = nullptr;
    int64_t ps_max = 0;   // largest per-colour sum of s^2 (the FP64 pivot workspace's size)
    double* d_pws = nullptr;
    int64_t* d_psoff = nullptr;
    int* d_boxes = nullptr;
    int* d_xoffs = nullptr;
    // double-float copies of the stored factors (precision IFMM_MIXED_SOLVE) and element counts
    int64_t npi = 0, ncp = 0, nbp = 0;
    dfl* d_Pi2 = nullptr;
    // digit slabs of the factors for the tensor-core replay (IFMM_MIXED_SOLVE with tc_products)
    uint8_t* d_slab = nullptr;
    int* d_srexp = nullptr;
    int64_t* d_soff = nullptr;
    int64_t* d_seoff = nullptr;
    dfl* d_Cp2 = nullptr;
    dfl* d_Bp2 = nullptr;
};

struct OpsLevel {
    std::vector<int> rank0;
    int* d_rank0 = nullptr;
    double* d_W0 = nullptr;
    double* d_Rt = nullptr;
    double* d_far0 = nullptr;
    // double-float copies for the inner matvec of IFMM_MIXED_SOLVE: W0 (used part) and far0
    int64_t nW0 = 0, nfar0 = 0;
    dfl* d_W0_2 = nullptr;
    dfl* d_far0_2 = nullptr;
};

uint64_t morton_host(Cell c, int dim) {
    uint64_t m = 0;
    for (int b = 0; b < 20; ++b) {
        m |= (uint64_t)((c.x >> b) & 1) << (dim * b);
        m |= (uint64_t)((c.y >> b) & 1) << (dim * b + 1);
        if (dim == 3) m |= (uint64_t)((c.z >> b) & 1) << (dim * b + 2);
    }
    return m;
}

}  // namespace

struct ifmm_handle {
    ifmm_params prm{};
    int kernel = 0;
    int device = 0;
    bool in_batch = false;   // factored by ifmm_factor_batch: pivot launches sized without a readback
    int64_t N = 0;
    int depth = 0, p = 0, r0 = 0, dim = 2;   // r0 = p^dim
    cudaStream_t st = nullptr;
    std::string err;
    std::vector<std::pair<void*, size_t>> allocs;
    cudaMemPool_t pool = nullptr;   // stream-ordered allocations on st (NULL: cudaMalloc / cudaFree)
    int64_t bytes = 0;
    // tree
    int64_t* d_perm = nullptr;
    double* d_px = nullptr;
    double* d_py = nullptr;
    double* d_pz = nullptr;   // zeros in 2D
    std::vector<int> leaf_count;
    std::vector<int64_t> leaf_start;
    int* d_leaf_count = nullptr;
    int64_t* d_leaf_start = nullptr;
    double* d_cheb = nullptr;
    double* d_Tc = nullptr;
    std::vector<OpsLevel> ops;
    std::vector<int64_t> p2p_off;
    int64_t* d_p2p_off = nullptr;
    double* d_p2p = nullptr;
    int64_t np2p = 0;
    dfl* d_p2p2 = nullptr;
    double sA = 0.0;
    // factor
    bool factored = false;
    std::vector<FLevel> lv;
    int M = 0;
    double* d_Dinv = nullptr;
    int* d_status = nullptr;
    double* d_counters = nullptr;
    // workspaces
    std::vector<std::pair<void*, size_t>> ws;
    ifmm_stats stats{};
};

namespace {

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                          \
            return e_ == cudaErrorMemoryAllocation ? IFMM_ERR_OOM : IFMM_ERR_CUDA;                \
        }                                                                                         \
    } while (0)

#define CKS(expr)                       \
    do {                                \
        ifmm_status s_ = (expr);        \
        if (s_ != IFMM_OK) return s_;   \
    } while (0)

// Every call on a handle runs with the handle's device current (the device that was current at
// ifmm_build) and gives the caller back the device it had: a caller that switched devices between
// calls must not have the kernels run on another GPU than the handle's memory.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) switched = cudaSetDevice(dev) == cudaSuccess;
        cudaGetLastError();
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

// Device memory of the handles comes from one library-owned, stream-ordered pool per device: buffers
// are allocated and freed in order on the handle's stream, so a free never synchronises the device
// (handles factored concurrently on separate streams keep overlapping), and the pool keeps freed
// memory for the next level or factorisation (release threshold unbounded; ifmm_destroy trims it).
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t library_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;
    } else {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pools[dev] = pool;
    return pool;
}

template <typename P>
ifmm_status dalloc(ifmm_handle* h, P** out, size_t bytes) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    cudaError_t e = h->pool ? cudaMallocFromPoolAsync(&p, bytes, h->pool, h->st) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? IFMM_ERR_OOM : IFMM_ERR_CUDA;
    }
    h->allocs.push_back({p, bytes});
    h->bytes += (int64_t)bytes;
    *out = static_cast<P*>(p);
    return IFMM_OK;
}

void dfree(ifmm_handle* h, void* p) {
    if (!p) return;
    for (size_t i = 0; i < h->allocs.size(); ++i)
        if (h->allocs[i].first == p) {
            h->bytes -= (int64_t)h->allocs[i].second;
            h->allocs.erase(h->allocs.begin() + i);
            if (h->pool) cudaFreeAsync(p, h->st);
            else cudaFree(p);
            return;
        }
}

template <typename P>
void dfree_ptr(ifmm_handle* h, P*& p) {
    dfree(h, (void*)p);
    p = nullptr;
}

template <typename V>
ifmm_status upload(ifmm_handle* h, typename V::value_type** out, const V& v) {
    CKS(dalloc(h, out, v.size() * sizeof(typename V::value_type)));
    if (!v.empty()) CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(typename V::value_type), cudaMemcpyHostToDevice, h->st));
    return IFMM_OK;
}

// growable named workspace
ifmm_status workspace(ifmm_handle* h, int slot, size_t bytes, void** out) {
    if ((int)h->ws.size() <= slot) h->ws.resize(slot + 1, {nullptr, 0});
    auto& w = h->ws[slot];
    if (w.second < bytes) {
        if (w.first) {
            CK(cudaStreamSynchronize(h->st));
            dfree(h, w.first);
        }
        w = {nullptr, 0};
        void* p = nullptr;
        CKS(dalloc(h, &p, bytes));
        w = {p, bytes};
    }
    *out = w.first;
    return IFMM_OK;
}

// ------------------------------------------------------------------------------------------------
// build
// ------------------------------------------------------------------------------------------------
ifmm_status do_build(ifmm_handle* h, const double* pts_host) {
    const int64_t N = h->N;
    const int dim = h->dim, nd = ndirs(dim), nk = 1 << dim;
    const int kap = h->depth, side = 1 << kap, nleaf = 1 << (dim * kap);
    const int p = h->p, r0 = h->r0;
    CKS(dalloc(h, &h->d_status, sizeof(int) * 4));
    CK(cudaMemsetAsync(h->d_status, 0, sizeof(int) * 4, h->st));
    CKS(dalloc(h, &h->d_counters, sizeof(double) * kCounters));
    CK(cudaMemsetAsync(h->d_counters, 0, sizeof(double) * kCounters, h->st));
    double* d_pts = nullptr;
    CKS(dalloc(h, &d_pts, sizeof(double) * dim * N));
    CK(cudaMemcpyAsync(d_pts, pts_host, sizeof(double) * dim * N, cudaMemcpyHostToDevice, h->st));
    int64_t npad = 1;
    while (npad < N) npad <<= 1;
    unsigned long long* d_keys = nullptr;
    CKS(dalloc(h, &d_keys, sizeof(unsigned long long) * npad));
    launch_leaf_keys(d_pts, N, kap, dim, h->prm.box[0], h->prm.box[1], h->prm.z0, h->prm.box[2], d_keys, npad,
                     h->d_status, h->st);
    launch_bitonic_sort(d_keys, npad, h->st);
    CKS(dalloc(h, &h->d_perm, sizeof(int64_t) * N));
    CKS(dalloc(h, &h->d_px, sizeof(double) * N));
    CKS(dalloc(h, &h->d_py, sizeof(double) * N));
    CKS(dalloc(h, &h->d_pz, sizeof(double) * N));
    CKS(dalloc(h, &h->d_leaf_count, sizeof(int) * nleaf));
    CK(cudaMemsetAsync(h->d_leaf_count, 0, sizeof(int) * nleaf, h->st));
    launch_scatter_sorted(d_keys, d_pts, N, dim, h->d_perm, h->d_px, h->d_py, h->d_pz, h->d_leaf_count, kap, h->st);
    int hstat = 0;
    h->leaf_count.assign(nleaf, 0);
    CK(cudaMemcpyAsync(h->leaf_count.data(), h->d_leaf_count, sizeof(int) * nleaf, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&hstat, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    dfree_ptr(h, d_keys);
    dfree_ptr(h, d_pts);
    if (hstat & DEV_ERR_RANGE) {
        h->err = "a point lies outside the root box";
        return IFMM_ERR_INVALID_ARG;
    }
    // leaf_start in Morton order (tree order of the sorted points)
    std::vector<std::pair<uint64_t, int>> mk(nleaf);
    for (int g = 0; g < nleaf; ++g) mk[g] = {morton_host(cell_of(g, side, dim), dim), g};
    std::sort(mk.begin(), mk.end());
    h->leaf_start.assign(nleaf, 0);
    int64_t acc = 0;
    int max_n = 0;
    for (auto& kv : mk) {
        h->leaf_start[kv.second] = acc;
        acc += h->leaf_count[kv.second];
        max_n = std::max(max_n, h->leaf_count[kv.second]);
    }
    CKS(upload(h, &h->d_leaf_start, h->leaf_start));
    // Chebyshev nodes and child transfers T_c[m', m] = S^parent_m(child node m'), 2^d of them
    std::vector<double> cheb(p), Tc((size_t)nk * r0 * r0);
    for (int m = 0; m < p; ++m) cheb[m] = std::cos((2.0 * m + 1.0) * M_PI / (2.0 * p));
    auto lag = [&](int m, double x) {
        double v = 1.0;
        for (int j = 0; j < p; ++j)
            if (j != m) v *= (x - cheb[j]) / (cheb[m] - cheb[j]);
        return v;
    };
    for (int c = 0; c < nk; ++c)
        for (int mc = 0; mc < r0; ++mc) {      // child node (mx, my, mz)
            const int mxyz[3] = {mc % p, (mc / p) % p, mc / (p * p)};
            for (int m = 0; m < r0; ++m) {     // parent basis function (nx, ny, nz)
                const int nxyz[3] = {m % p, (m / p) % p, m / (p * p)};
                double v = 1.0;
                for (int i = 0; i < dim; ++i) v *= lag(nxyz[i], 0.5 * (cheb[mxyz[i]] - 1.0) + ((c >> i) & 1));
                Tc[((size_t)c * r0 + mc) * r0 + m] = v;
            }
        }
    CKS(upload(h, &h->d_cheb, cheb));
    CKS(upload(h, &h->d_Tc, Tc));
    BuildArgs ba{N, kap, p, r0, h->kernel, h->prm.kparam[0], h->prm.diag, h->prm.box[0], h->prm.box[1], h->prm.box[2],
                 dim, h->prm.z0};
    h->ops.assign(kap + 1, OpsLevel());
    // SVD compression of the Chebyshev interpolation (svd_eps > 0): per level, top first, the kept
    // singular vectors U_k (r0 x r0 arrays, the first rsvd[k] columns used), freed after the build
    double* d_U = nullptr;
    double* d_sig = nullptr;
    int* d_rsvd = nullptr;
    double* d_svd_scr = nullptr;
    for (int k = 0; k < 16; ++k) h->stats.svd_ranks[k] = 0;
    if (h->prm.svd_eps > 0.0) {
        CKS(dalloc(h, &d_U, sizeof(double) * (size_t)(kap + 1) * r0 * r0));
        CKS(dalloc(h, &d_sig, sizeof(double) * (size_t)(kap + 1) * r0));
        CKS(dalloc(h, &d_rsvd, sizeof(int) * (size_t)(kap + 1)));
        CKS(dalloc(h, &d_svd_scr, sizeof(double) * svd_scratch_doubles(r0, dim)));
        for (int k = 2; k <= kap; ++k) {
            const bool top = k == 2;
            launch_svd_level(ba, k, h->prm.svd_eps, h->d_cheb, h->d_Tc, top ? nullptr : d_U + (size_t)(k - 1) * r0 * r0,
                             top ? nullptr : d_sig + (size_t)(k - 1) * r0, top ? nullptr : d_rsvd + (k - 1),
                             d_U + (size_t)k * r0 * r0, d_sig + (size_t)k * r0, d_rsvd + k, d_svd_scr, h->st);
        }
        std::vector<int> rs(kap + 1, 0);
        CK(cudaMemcpyAsync(rs.data(), d_rsvd, sizeof(int) * (kap + 1), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        for (int k = 2; k <= kap && k < 16; ++k) h->stats.svd_ranks[k] = rs[k];
    }
    auto Uk = [&](int k) -> const double* { return d_U ? d_U + (size_t)k * r0 * r0 : nullptr; };
    auto rk = [&](int k) -> const int* { return d_rsvd ? d_rsvd + k : nullptr; };
    // leaf bases (W0 allocation holds 2 scratch copies behind the basis)
    {
        OpsLevel& O = h->ops[kap];
        CKS(dalloc(h, &O.d_W0, sizeof(double) * 3 * (size_t)N * r0));
        CKS(dalloc(h, &O.d_Rt, sizeof(double) * (size_t)nleaf * r0 * r0));
        CKS(dalloc(h, &O.d_rank0, sizeof(int) * nleaf));
        launch_leaf_basis(ba, h->d_px, h->d_py, h->d_pz, h->d_leaf_start, h->d_leaf_count, h->d_cheb, O.d_W0, O.d_Rt,
                          O.d_rank0, max_n, Uk(kap), rk(kap), h->st);
        O.nW0 = (int64_t)N * r0;
    }
    for (int k = kap - 1; k >= 2; --k) {
        OpsLevel& O = h->ops[k];
        int nb = 1 << (dim * k);
        CKS(dalloc(h, &O.d_W0, sizeof(double) * 4 * (size_t)nb * nk * r0 * r0));
        CKS(dalloc(h, &O.d_Rt, sizeof(double) * (size_t)nb * r0 * r0));
        CKS(dalloc(h, &O.d_rank0, sizeof(int) * nb));
        launch_parent_basis(ba, k, h->ops[k + 1].d_Rt, h->ops[k + 1].d_rank0, h->d_Tc, O.d_W0, O.d_Rt, O.d_rank0,
                            Uk(k), rk(k), h->st);
        O.nW0 = (int64_t)nb * nk * r0 * r0;
    }
    for (int k = 2; k <= kap; ++k) {
        OpsLevel& O = h->ops[k];
        int nb = 1 << (dim * k);
        const int nreg = nregion(dim);
        CKS(dalloc(h, &O.d_far0, sizeof(double) * (size_t)nb * nreg * r0 * r0));
        CK(cudaMemsetAsync(O.d_far0, 0, sizeof(double) * (size_t)nb * nreg * r0 * r0, h->st));
        launch_m2l_build(ba, k, h->d_cheb, O.d_Rt, O.d_far0, h->st);
        O.nfar0 = (int64_t)nb * nreg * r0 * r0;
        O.rank0.assign(nb, 0);
        CK(cudaMemcpyAsync(O.rank0.data(), O.d_rank0, sizeof(int) * nb, cudaMemcpyDeviceToHost, h->st));
    }
    dfree_ptr(h, d_U);
    dfree_ptr(h, d_sig);
    dfree_ptr(h, d_rsvd);
    dfree_ptr(h, d_svd_scr);
    // leaf P2P
    h->p2p_off.assign((size_t)nleaf * nd, 0);
    int64_t po = 0;
    for (int g = 0; g < nleaf; ++g) {
        const Cell cg = cell_of(g, side, dim);
        for (int d = 0; d < nd; ++d) {
            const Cell cq = cell_dir(cg, d, dim);
            if (!cell_in(cq, side)) continue;
            h->p2p_off[(size_t)g * nd + d] = po;
            po += (int64_t)h->leaf_count[g] * h->leaf_count[cell_index(cq, side)];
        }
    }
    CKS(upload(h, &h->d_p2p_off, h->p2p_off));
    CKS(dalloc(h, &h->d_p2p, sizeof(double) * (size_t)std::max<int64_t>(po, 1)));
    double* d_sA = nullptr;
    CKS(dalloc(h, &d_sA, sizeof(double)));
    CK(cudaMemsetAsync(d_sA, 0, sizeof(double), h->st));
    launch_p2p_build(ba, h->d_px, h->d_py, h->d_pz, h->d_leaf_start, h->d_leaf_count, h->d_p2p_off, h->d_p2p, d_sA,
                     h->st);
    CK(cudaMemcpyAsync(&h->sA, d_sA, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    h->np2p = po;
    // double-float operator copies for the inner Krylov matvec of the mixed-precision solve
    if (h->prm.precision == IFMM_MIXED_SOLVE) {
        for (int k = 2; k <= kap; ++k) {
            OpsLevel& O = h->ops[k];
            CKS(dalloc(h, &O.d_W0_2, sizeof(dfl) * (size_t)O.nW0));
            launch_split_dfl(O.d_W0, O.d_W0_2, O.nW0, h->st);
            CKS(dalloc(h, &O.d_far0_2, sizeof(dfl) * (size_t)O.nfar0));
            launch_split_dfl(O.d_far0, O.d_far0_2, O.nfar0, h->st);
        }
        CKS(dalloc(h, &h->d_p2p2, sizeof(dfl) * (size_t)std::max<int64_t>(po, 1)));
        launch_split_dfl(h->d_p2p, h->d_p2p2, po, h->st);
    }
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    dfree_ptr(h, d_sA);
    return IFMM_OK;
}

// ------------------------------------------------------------------------------------------------
// factor
// ------------------------------------------------------------------------------------------------
template <typename T>
LevelView<T> view_of(ifmm_handle* h, FLevel& L) {
    LevelView<T> v{};
    v.k = L.k; v.side = L.side; v.nb = L.nb; v.RC = L.RC;
    v.dim = L.dim; v.nd = ndirs(L.dim); v.ctr = ndirs(L.dim) / 2; v.nreg = nregion(L.dim);
    v.nmax = 0;
    for (int b = 0; b < (int)L.n.size(); ++b) v.nmax = std::max(v.nmax, L.n[b]);
    v.n = L.d_n; v.r = L.d_r; v.voff = L.d_voff;
    v.boff = L.d_boff; v.bld = L.d_bld; v.blk = (T*)L.d_blk; v.W = (T*)L.d_W;
    v.pioff = L.d_pioff; v.pild = L.d_pild; v.Pi = (T*)L.d_Pi;
    v.cpoff = L.d_cpoff; v.Cp = (T*)L.d_Cp; v.bpoff = L.d_bpoff; v.Bp = (T*)L.d_Bp;
    v.xsoff = L.d_xsoff; v.xsld = L.d_xsld; v.Xs = (T*)L.d_Xs;
    v.fsoff = L.d_fsoff; v.Fs = (T*)L.d_Fs; v.Fs2 = (T*)L.d_Fs2;
    v.rsoff = L.d_rsoff; v.Rs = (T*)L.d_Rs;
    v.cwsoff = L.d_cwsoff; v.Cws = L.d_Cws;
    v.pws = L.d_pws; v.psoff = L.d_psoff;
    v.status = h->d_status; v.counters = h->d_counters;
    v.eps = h->prm.eps;
    v.sA = h->prm.tau_ref == 2 ? L.scale : h->sA;
    v.tau_ref = h->prm.tau_ref == 0 ? 0 : 1;
    v.symmetric = 1;   // every kernel of the library is radial, hence symmetric
    v.gemm_dfl = (std::is_same<T, double>::value && h->prm.precision == IFMM_MIXED_SOLVE) ? 1 : 0;
    v.gemm_tc = (v.gemm_dfl && h->prm.tc_products >= 2) ? 1 : 0;
    return v;
}

// The level as the replay (Algorithm 2) reads it: with T = dfl, the double-float copies of the
// FP64 factors; the replay touches only n, r, offsets and the Pi, C and B panels.
template <typename T>
LevelView<T> solve_view(ifmm_handle* h, FLevel& L) {
    LevelView<T> v = view_of<T>(h, L);
    if (std::is_same<T, double>::value && L.d_slab) {
        v.sl.slab = L.d_slab;
        v.sl.rexp = L.d_srexp;
        v.sl.soff = L.d_soff;
        v.sl.eoff = L.d_seoff;
    }
    if (std::is_same<T, dfl>::value) {
        v.Pi = (T*)L.d_Pi2;
        v.Cp = (T*)L.d_Cp2;
        v.Bp = (T*)L.d_Bp2;
        v.blk = nullptr; v.W = nullptr; v.Xs = nullptr; v.Fs = nullptr; v.Fs2 = nullptr; v.Rs = nullptr;
    }
    return v;
}

template <typename T>
ifmm_status setup_level(ifmm_handle* h, int k) {
    const int kap = h->depth, dim = h->dim, nd = ndirs(dim), ctr = nd / 2, nreg = nregion(dim), nk = 1 << dim;
    const int ncol = ncolours(dim);
    FLevel& L = h->lv[k];
    L.k = k; L.side = 1 << k; L.nb = 1 << (dim * k); L.dim = dim;
    const int s = L.side, nb = L.nb;
    const OpsLevel& O = h->ops[k];
    L.n.assign(nb, 0);
    L.r0 = O.rank0;
    L.r = O.rank0;
    if (k == kap) {
        L.n = h->leaf_count;
        L.voff.assign(nb + 1, 0);
        for (int b = 0; b < nb; ++b) L.voff[b] = h->leaf_start[b];
        L.voff[nb] = h->N;
        L.vtot = h->N;
    } else {
        FLevel& C = h->lv[k + 1];
        L.xoffs.assign((size_t)nb * (nk + 1), 0);
        for (int b = 0; b < nb; ++b) {
            const Cell cb = cell_of(b, s, dim);
            int off = 0;
            for (int c = 0; c < nk; ++c) {
                const int cg = cell_index(child_cell(cb, c), C.side);
                L.xoffs[(size_t)b * (nk + 1) + c] = off;
                off += C.r[cg];
            }
            L.xoffs[(size_t)b * (nk + 1) + nk] = off;
            L.n[b] = off;
        }
        L.voff.assign(nb + 1, 0);
        for (int b = 0; b < nb; ++b) L.voff[b + 1] = L.voff[b] + L.n[b];
        L.vtot = L.voff[nb];
        // children's y / z rows inside this level's vectors
        C.yoff.assign(C.nb, 0);
        for (int cg = 0; cg < C.nb; ++cg) {
            const Cell cc = cell_of(cg, C.side, dim);
            const int P = cell_index(Cell{cc.x >> 1, cc.y >> 1, cc.z >> 1}, s);
            const int c = (cc.x & 1) + 2 * (cc.y & 1) + 4 * (cc.z & 1);
            C.yoff[cg] = L.voff[P] + L.xoffs[(size_t)P * (nk + 1) + c];
        }
        CKS(upload(h, &C.d_yoff, C.yoff));
    }
    int maxn = 0;
    for (int b = 0; b < nb; ++b) maxn = std::max(maxn, L.n[b]);
    L.RC = h->prm.r_cap > 0 ? h->prm.r_cap : std::max(maxn, h->r0);
    std::vector<int> cap(nb);
    for (int b = 0; b < nb; ++b) cap[b] = std::min(L.n[b], L.RC);
    // blocks
    std::vector<int64_t> boff((size_t)nb * nreg, -1);
    std::vector<int> bld((size_t)nb * nreg, 0);
    int64_t bo = 0;
    for (int b = 0; b < nb; ++b) {
        const Cell cb = cell_of(b, s, dim);
        for (int j = 0; j < nreg; ++j) {
            const Cell cq = region_cell(cb, j, dim);
            if (!cell_in(cq, s)) continue;
            const int q = cell_index(cq, s);
            const bool nbr = cheb_dist(cq, cb) <= 1;
            int rows = nbr ? L.n[b] : cap[b], cols = nbr ? L.n[q] : cap[q];
            boff[(size_t)b * nreg + j] = bo;
            bld[(size_t)b * nreg + j] = cols;
            bo += (int64_t)rows * cols;
        }
    }
    // pivot inverses, panels
    std::vector<int64_t> pioff(nb), cpoff((size_t)nb * nd, 0), bpoff((size_t)nb * nd, 0), psoff(nb, 0);
    std::vector<int> pild(nb);
    int64_t pio = 0, cpo = 0, bpo = 0;
    L.smax = 0;
    for (int b = 0; b < nb; ++b) {
        int sm = L.n[b] + cap[b];
        L.smax = std::max(L.smax, sm);
        pioff[b] = pio;
        pild[b] = sm;
        pio += (int64_t)sm * sm;
        const Cell cb = cell_of(b, s, dim);
        for (int d = 0; d < nd; ++d) {
            const Cell cq = cell_dir(cb, d, dim);
            if (d == ctr || !cell_in(cq, s)) continue;
            const int q = cell_index(cq, s);
            cpoff[(size_t)b * nd + d] = cpo;
            cpo += (int64_t)L.n[q] * L.n[b];
            bpoff[(size_t)b * nd + d] = bpo;
            bpo += (int64_t)L.n[b] * L.n[q];
        }
    }
    // colour lists (Morton order inside a colour). An empty box (n = 0, hence r = 0) has nothing
    // to eliminate: its pivot, panels and Schur, compression and redirect contributions are all of
    // size zero, so it is left out of the lists (uniform trees of clustered clouds are mostly empty)
    std::vector<std::pair<uint64_t, int>> keys;
    keys.reserve(nb);
    for (int b = 0; b < nb; ++b) {
        if (L.n[b] == 0) continue;
        const Cell cb = cell_of(b, s, dim);
        keys.push_back({((uint64_t)cell_colour(cb) << 58) | morton_host(cb, dim), b});
    }
    std::sort(keys.begin(), keys.end());
    const int nact = (int)keys.size();
    L.boxes.resize(nact);
    for (int t = 0; t < nact; ++t) L.boxes[t] = keys[t].second;
    for (int c = 0; c <= ncol; ++c) L.cstart[c] = 0;
    {
        int t = 0;
        for (int c = 0; c < ncol; ++c) {
            L.cstart[c] = t;
            while (t < nact && (int)(keys[t].first >> 58) == c) ++t;
        }
        L.cstart[ncol] = nact;
    }
    // per-colour scratch
    std::vector<int64_t> xsoff(nb, 0), fsoff((size_t)nb * nd * nd, 0), rsoff((size_t)nb * nd, 0),
        cwsoff((size_t)nb * nd, 0);
    std::vector<int> xsld(nb, 0);
    int64_t xs_max = 0, fs_max = 0, rs_max = 0, ps_max = 0, cw_max = 0;
    for (int c = 0; c < ncol; ++c) {
        int64_t xo = 0, fo = 0, ro = 0, pso = 0, cwo = 0;
        for (int t = L.cstart[c]; t < L.cstart[c + 1]; ++t) {
            const int e = L.boxes[t];
            const Cell ce = cell_of(e, s, dim);
            int sm = L.n[e] + cap[e];
            int ld = cap[e];
            for (int d = 0; d < nd; ++d) {
                const Cell cq = cell_dir(ce, d, dim);
                if (d == ctr || !cell_in(cq, s)) continue;
                ld += L.n[cell_index(cq, s)];
            }
            xsoff[e] = xo;
            xsld[e] = ld;
            xo += (int64_t)sm * ld;
            psoff[e] = pso;
            pso += (int64_t)sm * sm;
            for (int dp = 0; dp < nd; ++dp)
                for (int dq = 0; dq < nd; ++dq) {
                    const Cell cp = cell_dir(ce, dp, dim), cq = cell_dir(ce, dq, dim);
                    if (dp == ctr || dq == ctr || !cell_in(cp, s) || !cell_in(cq, s)) continue;
                    if (cheb_dist(cp, cq) != 2) continue;
                    fsoff[((size_t)e * nd + dp) * nd + dq] = fo;
                    fo += (int64_t)L.n[cell_index(cp, s)] * L.n[cell_index(cq, s)];
                }
            for (int dq = 0; dq < nd; ++dq) {
                const Cell cq = cell_dir(ce, dq, dim);
                if (dq == ctr || !cell_in(cq, s)) continue;
                int64_t mb = 0;
                for (int dp = 0; dp < nd; ++dp) {
                    const Cell cp = cell_dir(ce, dp, dim);
                    if (dp == ctr || !cell_in(cp, s)) continue;
                    if (cheb_dist(cp, cq) == 2) mb += 2 * L.n[cell_index(cp, s)];
                }
                const int nq = L.n[cell_index(cq, s)];
                rsoff[(size_t)e * nd + dq] = ro;
                ro += (int64_t)nq * mb;
                // the compression's work arrays: the basis vector (n_q), 8 x RC coefficients, m norms,
                // the basis vector again in the column arithmetic's type (n_q)
                cwsoff[(size_t)e * nd + dq] = cwo;
                cwo += 2 * (int64_t)nq + 8 * (int64_t)L.RC + mb;
            }
        }
        xs_max = std::max(xs_max, xo);
        fs_max = std::max(fs_max, fo);
        rs_max = std::max(rs_max, ro);
        cw_max = std::max(cw_max, cwo);
        ps_max = std::max(ps_max, pso);
    }
    size_t es = sizeof(T);
    CKS(upload(h, &L.d_n, L.n));
    CKS(upload(h, &L.d_r, L.r));
    CKS(upload(h, &L.d_voff, L.voff));
    CKS(upload(h, &L.d_boff, boff));
    CKS(upload(h, &L.d_bld, bld));
    CKS(dalloc(h, &L.d_blk, es * (size_t)bo));
    CK(cudaMemsetAsync(L.d_blk, 0, es * (size_t)bo, h->st));
    CKS(dalloc(h, &L.d_W, es * (size_t)L.vtot * L.RC));
    CK(cudaMemsetAsync(L.d_W, 0, es * (size_t)L.vtot * L.RC, h->st));
    CKS(upload(h, &L.d_pioff, pioff));
    CKS(upload(h, &L.d_pild, pild));
    CKS(dalloc(h, &L.d_Pi, es * (size_t)pio));
    L.npi = pio;
    CKS(upload(h, &L.d_cpoff, cpoff));
    CKS(dalloc(h, &L.d_Cp, es * (size_t)cpo));
    L.ncp = cpo;
    CKS(upload(h, &L.d_bpoff, bpoff));
    CKS(dalloc(h, &L.d_Bp, es * (size_t)bpo));
    L.nbp = bpo;
    CKS(upload(h, &L.d_xsoff, xsoff));
    CKS(upload(h, &L.d_xsld, xsld));
    CKS(dalloc(h, &L.d_Xs, es * (size_t)xs_max));
    CKS(upload(h, &L.d_fsoff, fsoff));
    CKS(dalloc(h, &L.d_Fs, es * (size_t)fs_max));
    CKS(dalloc(h, &L.d_Fs2, es * (size_t)fs_max));
    CKS(upload(h, &L.d_rsoff, rsoff));
    CKS(dalloc(h, &L.d_Rs, es * (size_t)rs_max));
    CKS(upload(h, &L.d_cwsoff, cwsoff));
    CKS(dalloc(h, &L.d_Cws, sizeof(double) * (size_t)std::max<int64_t>(cw_max, 1)));
    CKS(upload(h, &L.d_psoff, psoff));
    // FP64 pivot workspace in global memory for blocks whose matrix does not fit in shared memory
    // (single block per box) or whose cluster slabs do not (8-block clusters)
    L.ps_max = ps_max;
    if ((size_t)L.smax * L.smax * 8 > 150 * 1024) CKS(dalloc(h, &L.d_pws, sizeof(double) * (size_t)ps_max));
    CKS(upload(h, &L.d_boxes, L.boxes));
    if (k < kap) CKS(upload(h, &L.d_xoffs, L.xoffs));
    LevelView<T> v = view_of<T>(h, L);
    if (k == kap) {
        launch_init_level<T>(v, 1, h->d_p2p, h->d_p2p_off, O.d_W0, h->d_leaf_start, h->r0, nullptr, O.d_far0,
                             O.d_rank0, nullptr, nullptr, h->st);
    } else {
        LevelView<T> cv = view_of<T>(h, h->lv[k + 1]);
        launch_init_level<T>(v, 0, nullptr, nullptr, O.d_W0, nullptr, h->r0, L.d_xoffs, O.d_far0, O.d_rank0,
                             h->ops[k + 1].d_rank0, &cv, h->st);
    }
    // threshold reference of the level: largest column norm of its diagonal blocks
    double* d_sc = nullptr;
    CKS(dalloc(h, &d_sc, sizeof(double)));
    CK(cudaMemsetAsync(d_sc, 0, sizeof(double), h->st));
    launch_level_scale<T>(v, d_sc, h->st);
    CK(cudaMemcpyAsync(&L.scale, d_sc, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    dfree_ptr(h, d_sc);
    CK(cudaGetLastError());
    return IFMM_OK;
}

template <typename T>
void free_level_work(ifmm_handle* h, FLevel& L) {
    dfree_ptr(h, L.d_blk);
    dfree_ptr(h, L.d_W);
    dfree_ptr(h, L.d_Xs);
    dfree_ptr(h, L.d_Fs);
    dfree_ptr(h, L.d_Fs2);
    dfree_ptr(h, L.d_Rs);
    dfree_ptr(h, L.d_Cws);
    dfree_ptr(h, L.d_pws);
}

void release_level(ifmm_handle* h, FLevel& L) {
    void** ptrs[] = {(void**)&L.d_n, (void**)&L.d_r, (void**)&L.d_voff, (void**)&L.d_yoff, (void**)&L.d_boff,
                     (void**)&L.d_bld, &L.d_blk, &L.d_W, (void**)&L.d_pioff, (void**)&L.d_pild, &L.d_Pi,
                     (void**)&L.d_cpoff, &L.d_Cp, (void**)&L.d_bpoff, &L.d_Bp, (void**)&L.d_xsoff,
                     (void**)&L.d_xsld, &L.d_Xs, (void**)&L.d_fsoff, &L.d_Fs, &L.d_Fs2, (void**)&L.d_rsoff,
                     &L.d_Rs, (void**)&L.d_cwsoff, (void**)&L.d_Cws, (void**)&L.d_pws, (void**)&L.d_psoff, (void**)&L.d_boxes, (void**)&L.d_xoffs,
                     (void**)&L.d_Pi2, (void**)&L.d_Cp2, (void**)&L.d_Bp2, (void**)&L.d_slab, (void**)&L.d_srexp,
                     (void**)&L.d_soff, (void**)&L.d_seoff};
    for (void** p : ptrs) {
        dfree(h, *p);
        *p = nullptr;
    }
}

// discard a previous factorisation (device memory and host tables)
void release_factors(ifmm_handle* h) {
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    for (auto& L : h->lv) release_level(h, L);
    h->lv.clear();
    dfree_ptr(h, h->d_Dinv);
    h->M = 0;
    h->factored = false;
}

// double-float copies of the FP64 factors for the replay of IFMM_MIXED_SOLVE (the level-1 inverse
// stays FP64)
ifmm_status split_factors(ifmm_handle* h) {
    for (int k = 2; k <= h->depth; ++k) {
        FLevel& L = h->lv[k];
        CKS(dalloc(h, &L.d_Pi2, sizeof(dfl) * (size_t)std::max<int64_t>(L.npi, 1)));
        launch_split_dfl((const double*)L.d_Pi, L.d_Pi2, L.npi, h->st);
        CKS(dalloc(h, &L.d_Cp2, sizeof(dfl) * (size_t)std::max<int64_t>(L.ncp, 1)));
        launch_split_dfl((const double*)L.d_Cp, L.d_Cp2, L.ncp, h->st);
        CKS(dalloc(h, &L.d_Bp2, sizeof(dfl) * (size_t)std::max<int64_t>(L.nbp, 1)));
        launch_split_dfl((const double*)L.d_Bp, L.d_Bp2, L.nbp, h->st);
    }
    CK(cudaGetLastError());
    return IFMM_OK;
}

// Digit slabs of every level's factors for the tensor-core replay (IFMM_MIXED_SOLVE, tc_products): the
// operands of the replay's products split once (ifmm_tc.cuh), twelve per box (kSlabRecs): Pi with
// rows s and K = n, Pi with rows n and K = s, the C panel of each neighbour direction (rows = the
// neighbour's width at the elimination, K = n) and the B panels side by side (rows n, K = the sum of
// the widths). Record sizes follow tc::slab_bytes; the host lays the records out per level.
ifmm_status presplit_factors(ifmm_handle* h) {
    for (int k = 2; k <= h->depth; ++k) {
        FLevel& L = h->lv[k];
        const int s = L.side;
        std::vector<int64_t> soff((size_t)L.nb * kSlabRecs, -1), eoff((size_t)L.nb * kSlabRecs, 0);
        int64_t bytes = 0, exps = 0;
        auto add = [&](int e, int rec, int rows, int K) {
            if (rows <= 0 || K <= 0) return;
            soff[(size_t)e * kSlabRecs + rec] = bytes;
            eoff[(size_t)e * kSlabRecs + rec] = exps;
            bytes += tc::slab_bytes(rows, K);
            exps += (int64_t)((rows + 7) / 8) * 8;
        };
        for (int e : L.boxes) {
            const int n = L.n[e], r = L.r[e], ex = e % s, ey = e / s, ce = (ex % 3) + 3 * (ey % 3);
            add(e, 0, n + r, n);
            add(e, 1, n, n + r);
            int ksum = 0;
            for (int d = 0; d < 9; ++d) {
                const int qx = ex + d % 3 - 1, qy = ey + d / 3 - 1;
                if (d == 4 || qx < 0 || qy < 0 || qx >= s || qy >= s) continue;
                const int q = qx + s * qy, cq = (qx % 3) + 3 * (qy % 3);
                const int w = cq < ce ? L.r[q] : L.n[q];
                add(e, 2 + d, w, n);
                ksum += w;
            }
            add(e, 11, n, ksum);
        }
        CKS(dalloc(h, &L.d_slab, (size_t)std::max<int64_t>(bytes, 16)));
        CKS(dalloc(h, &L.d_srexp, sizeof(int) * (size_t)std::max<int64_t>(exps, 1)));
        CKS(upload(h, &L.d_soff, soff));
        CKS(upload(h, &L.d_seoff, eoff));
        LevelView<double> v = view_of<double>(h, L);
        v.sl.soff = L.d_soff;
        v.sl.eoff = L.d_seoff;
        for (int c = 0; c < 9; ++c)
            launch_presplit(v, L.d_slab, L.d_srexp, L.d_boxes + L.cstart[c], L.cstart[c + 1] - L.cstart[c], c, h->st);
    }
    CK(cudaGetLastError());
    return IFMM_OK;
}

// A factorisation in phases, so that a batch of systems can run its levels in lockstep (factor_fused):
// factor_begin; per level k = depth..2: factor_level_setup, the colours' launches, factor_level_end;
// factor_finish (the level-1 system). factor_impl runs them for one system.
template <typename T>
ifmm_status factor_begin(ifmm_handle* h) {
    h->lv.assign(h->depth + 1, FLevel());
    CK(cudaMemsetAsync(h->d_status, 0, sizeof(int) * 4, h->st));
    CK(cudaMemsetAsync(h->d_counters, 0, sizeof(double) * kCounters, h->st));
    for (int k = 0; k < 16; ++k) h->stats.level_ms[k] = 0.0;
    for (int t = 0; t < 5; ++t) {
        h->stats.kernel_ms[t] = 0.0;
        h->stats.kernel_launches[t] = 0;
    }
    return IFMM_OK;
}

template <typename T>
ifmm_status factor_level_setup(ifmm_handle* h, int k) {
    CKS(setup_level<T>(h, k));
    if (k < h->depth) {
        CK(cudaStreamSynchronize(h->st));
        free_level_work<T>(h, h->lv[k + 1]);
    }
    return IFMM_OK;
}

// status and ranks of level k after its colours ran (a stream synchronisation)
template <typename T>
ifmm_status factor_level_end(ifmm_handle* h, int k) {
    FLevel& L = h->lv[k];
    CK(cudaGetLastError());
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(L.r.data(), L.d_r, sizeof(int) * L.nb, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (hs & DEV_ERR_SINGULAR) {
        h->err = "singular pivot block at level " + std::to_string(k);
        return IFMM_ERR_SINGULAR_PIVOT;
    }
    if (hs & DEV_ERR_TIMEOUT) {
        h->err = "a bounded wait on the tensor cores ran out at level " + std::to_string(k);
        return IFMM_ERR_TIMEOUT;
    }
    if (hs & DEV_ERR_SIZE) {
        h->err = "the well-separated fill at level " + std::to_string(k) +
                 " is wider than the compression's shared-memory arrays";
        return IFMM_ERR_INVALID_ARG;
    }
    return IFMM_OK;
}

template <typename T>
ifmm_status factor_finish(ifmm_handle* h, long long l0) {
    // level 1: dense system over the level-2 multipoles
    FLevel& L2 = h->lv[2];
    L2.yoff.assign(L2.nb, 0);
    int64_t M = 0;
    for (int b = 0; b < L2.nb; ++b) {
        L2.yoff[b] = M;
        M += L2.r[b];
    }
    h->M = (int)M;
    CKS(upload(h, &L2.d_yoff, L2.yoff));
    CKS(dalloc(h, &h->d_Dinv, sizeof(double) * (size_t)std::max<int64_t>(M * M, 1)));
    CK(cudaMemsetAsync(h->d_Dinv, 0, sizeof(double) * (size_t)M * M, h->st));
    LevelView<T> v2 = view_of<T>(h, L2);
    launch_root_gather<T>(v2, L2.d_yoff, h->d_Dinv, (int)M, h->st);
    int* d_perm = nullptr;
    double* d_col = nullptr;
    CKS(dalloc(h, &d_perm, sizeof(int) * (size_t)(M + 1)));
    CKS(dalloc(h, &d_col, sizeof(double) * (size_t)(M + 1)));
    launch_dense_invert(h->d_Dinv, (int)M, d_perm, d_col, h->d_status, h->st);
    int hs = 0;
    double cnt[kCounters];
    CK(cudaMemcpyAsync(&hs, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(cnt, h->d_counters, sizeof(double) * kCounters, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    dfree_ptr(h, d_perm);
    dfree_ptr(h, d_col);
    free_level_work<T>(h, L2);
    if (hs & DEV_ERR_SINGULAR) {
        h->err = "singular level-1 system";
        return IFMM_ERR_SINGULAR_PIVOT;
    }
    int maxr = 0;
    for (int k = 2; k <= h->depth; ++k)
        for (int b = 0; b < h->lv[k].nb; ++b) maxr = std::max(maxr, h->lv[k].r[b]);
    h->stats.max_rank = maxr;
    h->stats.schur_flops = cnt[0];
    h->stats.schur_bytes = cnt[1];
    h->stats.factor_flops = cnt[2] + 2.0 * (double)M * M * M;
    const int fidx[5] = {3, 4, 0, 5, 6};
    for (int t = 0; t < 5; ++t) h->stats.kernel_flops[t] = cnt[fidx[t]];
    h->stats.compress_proj_flops = cnt[7];
    h->stats.compress_reorth_flops = cnt[8];
    h->stats.launches_factor = launches_so_far() - l0;
    h->stats.rank_overflows = 0;
    h->factored = true;
    if (hs & DEV_ERR_OVERFLOW) {
        h->stats.rank_overflows = 1;
        h->err = "a box basis reached r_cap; the factorisation is usable but coarser than eps";
        return IFMM_ERR_RANK_OVERFLOW;
    }
    return IFMM_OK;
}

template <typename T>
ifmm_status factor_impl(ifmm_handle* h) {
    const int kap = h->depth;
    CKS(factor_begin<T>(h));
    const long long l0 = launches_so_far();
    const int ncol = ncolours(h->dim);
    std::vector<cudaEvent_t> ev(ncol * 6);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    struct EvGuard {
        std::vector<cudaEvent_t>& v;
        ~EvGuard() { for (auto e : v) cudaEventDestroy(e); }
    } evg{ev};
    for (int k = kap; k >= 2; --k) {
        CKS(factor_level_setup<T>(h, k));
        FLevel& L = h->lv[k];
        LevelView<T> v = view_of<T>(h, L);
        bool used[27] = {false};
        for (int c = 0; c < ncol; ++c) {
            int cnt = L.cstart[c + 1] - L.cstart[c];
            if (cnt <= 0) continue;
            launch_factor_colour<T>(v, L.d_boxes + L.cstart[c], cnt, c, L.smax, h->in_batch ? 0 : 1, h->st,
                                    &ev[c * 6]);
            used[c] = true;
        }
        CKS(factor_level_end<T>(h, k));
        double lms = 0.0;
        for (int c = 0; c < ncol; ++c) {
            if (!used[c]) continue;
            for (int t = 0; t < 5; ++t) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ev[c * 6 + t], ev[c * 6 + t + 1]));
                h->stats.kernel_ms[t] += ms;
                h->stats.kernel_launches[t] += 1;
                lms += ms;
            }
        }
        if (k < 16) h->stats.level_ms[k] = lms;
    }
    return factor_finish<T>(h, l0);
}

// Worker threads run one function per system (index i of `idx`); returns after all finished.
template <class F>
void for_each_system(const std::vector<int>& idx, int workers, F fn) {
    if (idx.empty()) return;
    workers = std::max(1, std::min<int>(workers, (int)idx.size()));
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    for (int w = 0; w < workers; ++w)
        pool.emplace_back([&]() {
            for (int t; (t = next.fetch_add(1)) < (int)idx.size();) fn(idx[t]);
        });
    for (auto& t : pool) t.join();
}

// Batched factorisation in lockstep (no counterpart in the paper, which eliminates one system):
// step t eliminates level depth_s - t of every system s that has it, and every colour of that step is
// one launch of each factor kernel over the boxes of all those systems together (a global list of
// (system, box) items; each block reads its system's level view from device memory), on the
// batch's own stream. Per-system work (level set-up, status and rank read-back, the level-1 system)
// runs on the systems' streams in worker threads. Same device and precision for every handle.
template <typename T>
ifmm_status factor_fused(ifmm_h* hs, int n, int workers, ifmm_status* st_out) {
    std::vector<ifmm_status> st(n, IFMM_OK);
    const int dev = hs[0]->device;
    cudaStream_t B = nullptr;
    if (cudaStreamCreateWithFlags(&B, cudaStreamNonBlocking) != cudaSuccess) return IFMM_ERR_CUDA;
    std::vector<cudaEvent_t> evs(n, nullptr);
    cudaEvent_t evB = nullptr;
    cudaEventCreateWithFlags(&evB, cudaEventDisableTiming);
    for (auto& e : evs) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    const long long l0 = launches_so_far();
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    auto on_dev = [&](auto fn) { return [&, fn](int i) { cudaSetDevice(dev); fn(i); }; };
    for_each_system(all, workers, on_dev([&](int i) {
        hs[i]->err.clear();
        release_factors(hs[i]);
        st[i] = factor_begin<T>(hs[i]);
    }));
    int maxd = 0;
    for (int i = 0; i < n; ++i) maxd = std::max(maxd, hs[i]->depth);
    ifmm_handle* h0 = hs[0];
    for (int t = 0; maxd - t >= 2; ++t) {
        std::vector<int> act;
        for (int i = 0; i < n; ++i)
            if (st[i] == IFMM_OK && hs[i]->depth - t >= 2) act.push_back(i);
        if (act.empty()) break;
        for_each_system(act, workers, on_dev([&](int i) {
            ifmm_handle* h = hs[i];
            st[i] = factor_level_setup<T>(h, h->depth - t);
            if (st[i] == IFMM_OK) cudaEventRecord(evs[i], h->st);
        }));
        std::vector<int> ok;
        for (int i : act)
            if (st[i] == IFMM_OK) ok.push_back(i);
        if (ok.empty()) continue;
        // launch sizes over the batch: the largest pivot, box and rank cap
        int smax = 0, nmax = 0, rc = 0, rep = ok[0];
        for (int i : ok) {
            const FLevel& L = hs[i]->lv[hs[i]->depth - t];
            if (L.smax > smax) { smax = L.smax; rep = i; }
            for (int b : L.boxes) nmax = std::max(nmax, L.n[b]);
            rc = std::max(rc, L.RC);
        }
        // blocks whose pivot slab lives in the FP64 workspace need it in every system of the launch
        if ((size_t)smax * smax * 8 > 150 * 1024)
            for (int i : ok) {
                FLevel& L = hs[i]->lv[hs[i]->depth - t];
                if (!L.d_pws && dalloc(hs[i], &L.d_pws, sizeof(double) * (size_t)std::max<int64_t>(L.ps_max, 1)) != IFMM_OK)
                    st[i] = IFMM_ERR_OOM;
                cudaEventRecord(evs[i], hs[i]->st);
            }
        std::vector<LevelView<T>> views;
        std::vector<int> vi(n, -1);
        for (int i : ok) {
            if (st[i] != IFMM_OK) continue;
            vi[i] = (int)views.size();
            views.push_back(view_of<T>(hs[i], hs[i]->lv[hs[i]->depth - t]));
        }
        if (views.empty()) continue;
        std::vector<int2> items;
        const int ncol = ncolours(hs[0]->dim);
        int cstart[28];
        for (int c = 0; c < ncol; ++c) {
            cstart[c] = (int)items.size();
            for (int i : ok) {
                if (vi[i] < 0) continue;
                const FLevel& L = hs[i]->lv[hs[i]->depth - t];
                for (int q = L.cstart[c]; q < L.cstart[c + 1]; ++q) items.push_back(make_int2(vi[i], L.boxes[q]));
            }
        }
        cstart[ncol] = (int)items.size();
        for (int i : ok)
            if (vi[i] >= 0) cudaStreamWaitEvent(B, evs[i], 0);
        LevelView<T>* d_views = nullptr;
        int2* d_items = nullptr;
        ifmm_status s0 = IFMM_OK;
        if (cudaMallocAsync((void**)&d_views, sizeof(LevelView<T>) * views.size(), B) != cudaSuccess ||
            cudaMallocAsync((void**)&d_items, sizeof(int2) * std::max<size_t>(items.size(), 1), B) != cudaSuccess)
            s0 = IFMM_ERR_OOM;
        if (s0 == IFMM_OK) {
            cudaMemcpyAsync(d_views, views.data(), sizeof(LevelView<T>) * views.size(), cudaMemcpyHostToDevice, B);
            cudaMemcpyAsync(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, B);
            LevelView<T> Lr = views[vi[rep] >= 0 ? vi[rep] : 0];
            Lr.nmax = nmax;
            Lr.RC = rc;
            for (int c = 0; c < ncol; ++c) {
                const int cnt = cstart[c + 1] - cstart[c];
                if (cnt > 0)
                    launch_factor_colour<T>(Lr, nullptr, cnt, c, smax, 0, B, nullptr, d_items + cstart[c], d_views);
            }
            cudaFreeAsync(d_views, B);
            cudaFreeAsync(d_items, B);
        }
        cudaEventRecord(evB, B);
        for_each_system(ok, workers, on_dev([&](int i) {
            if (st[i] != IFMM_OK) return;
            ifmm_handle* h = hs[i];
            if (s0 != IFMM_OK) {
                st[i] = s0;
                return;
            }
            cudaStreamWaitEvent(h->st, evB, 0);
            st[i] = factor_level_end<T>(h, h->depth - t);
        }));
    }
    for_each_system(all, workers, on_dev([&](int i) {
        if (st[i] == IFMM_OK) st[i] = factor_finish<T>(hs[i], l0);
        if (st[i] != IFMM_OK && st[i] != IFMM_ERR_RANK_OVERFLOW) hs[i]->factored = false;
    }));
    cudaStreamSynchronize(B);
    cudaStreamDestroy(B);
    cudaEventDestroy(evB);
    for (auto& e : evs) cudaEventDestroy(e);
    ifmm_status first = IFMM_OK;
    for (int i = 0; i < n; ++i) {
        if (st_out) st_out[i] = st[i];
        if (first == IFMM_OK && st[i] != IFMM_OK) first = st[i];
    }
    return first;
}

// ------------------------------------------------------------------------------------------------
// solve
// ------------------------------------------------------------------------------------------------
// in: tree-order rhs (vtot_kappa x nrhs, T) in workspace 0 ; out: tree-order x in workspace 1
template <typename T>
ifmm_status solve_core(ifmm_handle* h, int nrhs, T* rhs_leaf, T* x_leaf) {
    const int kap = h->depth;
    std::vector<T*> vr(kap + 1, nullptr), vx(kap + 1, nullptr);
    vr[kap] = rhs_leaf;
    vx[kap] = x_leaf;
    int64_t maxv = 0;
    for (int k = kap; k >= 2; --k) maxv = std::max(maxv, h->lv[k].vtot);
    // workspace slots: 2.. hold the level vectors
    int slot = 2;
    for (int k = kap - 1; k >= 1; --k) {
        int64_t len = (k >= 2) ? h->lv[k].vtot : h->M;
        void* p1 = nullptr;
        void* p2 = nullptr;
        CKS(workspace(h, slot++, sizeof(T) * (size_t)std::max<int64_t>(len * nrhs, 1), &p1));
        CKS(workspace(h, slot++, sizeof(T) * (size_t)std::max<int64_t>(len * nrhs, 1), &p2));
        vr[k] = (T*)p1;
        vx[k] = (T*)p2;
    }
    void* pv = nullptr;
    CKS(workspace(h, slot++, sizeof(T) * (size_t)std::max<int64_t>(maxv * nrhs, 1), &pv));
    T* vxs = (T*)pv;
    // split-K scratch of the back substitution at the upper levels (partials and tile counters)
    const int64_t part_cap = (int64_t)4 << 20;
    const int cnt_cap = 4096;
    void *pp = nullptr, *pc = nullptr;
    CKS(workspace(h, 26, sizeof(T) * (size_t)part_cap, &pp));
    CKS(workspace(h, 27, sizeof(int) * (size_t)cnt_cap, &pc));
    CK(cudaMemsetAsync(pc, 0, sizeof(int) * (size_t)cnt_cap, h->st));
    for (int k = kap; k >= 2; --k) {
        FLevel& L = h->lv[k];
        LevelView<T> v = solve_view<T>(h, L);
        for (int c = 0; c < ncolours(h->dim); ++c) {
            int cnt = L.cstart[c + 1] - L.cstart[c];
            launch_forward_colour<T>(v, L.d_boxes + L.cstart[c], cnt, c, L.d_yoff, vr[k], vr[k - 1], vxs, nrhs, h->st);
        }
    }
    launch_root_apply<T>(h->d_Dinv, h->M, vr[1], vx[1], nrhs, h->st);
    for (int k = 2; k <= kap; ++k) {
        FLevel& L = h->lv[k];
        LevelView<T> v = solve_view<T>(h, L);
        for (int c = ncolours(h->dim) - 1; c >= 0; --c) {
            int cnt = L.cstart[c + 1] - L.cstart[c];
            launch_backward_colour<T>(v, L.d_boxes + L.cstart[c], cnt, c, L.d_yoff, vr[k], vx[k], vx[k - 1], vxs,
                                      nrhs, (T*)pp, part_cap, (int*)pc, cnt_cap, h->st);
        }
    }
    CK(cudaGetLastError());
    return IFMM_OK;
}

template <typename T>
ifmm_status solve_once(ifmm_handle* h, const double* b, int64_t ldb, double* x, int64_t ldx, int nrhs) {
    void* p0 = nullptr;
    void* p1 = nullptr;
    CKS(workspace(h, 0, sizeof(T) * (size_t)h->N * nrhs, &p0));
    CKS(workspace(h, 1, sizeof(T) * (size_t)h->N * nrhs, &p1));
    launch_permute_in<T>(b, ldb, h->N, nrhs, h->d_perm, (T*)p0, h->st);
    CKS(solve_core<T>(h, nrhs, (T*)p0, (T*)p1));
    launch_permute_out<T>((T*)p1, h->N, nrhs, h->d_perm, x, ldx, h->st);
    CK(cudaGetLastError());
    return IFMM_OK;
}

ifmm_status matvec_impl(ifmm_handle* h, const double* x, int64_t ldx, double* y, int64_t ldy, int nrhs) {
    const int kap = h->depth, r0 = h->r0;
    void* pxt = nullptr;
    void* pout = nullptr;
    CKS(workspace(h, 40, sizeof(double) * (size_t)h->N * nrhs, &pxt));
    CKS(workspace(h, 41, sizeof(double) * (size_t)h->N * nrhs, &pout));
    double* xt = (double*)pxt;
    double* out = (double*)pout;
    std::vector<double*> ym(kap + 1, nullptr), zm(kap + 1, nullptr);
    for (int k = 2; k <= kap; ++k) {
        size_t len = sizeof(double) * ((size_t)1 << (h->dim * k)) * r0 * nrhs;
        void* a = nullptr;
        void* b = nullptr;
        CKS(workspace(h, 120 + 2 * k, len, &a));
        CKS(workspace(h, 121 + 2 * k, len, &b));
        ym[k] = (double*)a;
        zm[k] = (double*)b;
    }
    launch_mv_permute_in(x, ldx, h->N, nrhs, h->d_perm, xt, h->st);
    launch_mv_leaf_up(h->dim, kap, h->ops[kap].d_W0, h->d_leaf_start, h->d_leaf_count, r0, xt, ym[kap], nrhs, h->st);
    for (int k = kap - 1; k >= 2; --k) launch_mv_up(h->dim, k, h->ops[k].d_W0, r0, ym[k + 1], ym[k], nrhs, h->st);
    for (int k = 2; k <= kap; ++k) launch_mv_m2l(h->dim, k, h->ops[k].d_far0, r0, ym[k], zm[k], nrhs, h->st);
    for (int k = 2; k < kap; ++k) launch_mv_down(h->dim, k, h->ops[k].d_W0, r0, zm[k], zm[k + 1], nrhs, h->st);
    launch_mv_leaf_down(h->dim, kap, h->ops[kap].d_W0, h->d_leaf_start, h->d_leaf_count, r0, zm[kap], xt, h->d_p2p_off,
                        h->d_p2p, out, nrhs, h->st);
    launch_mv_permute_out(out, h->N, nrhs, h->d_perm, y, ldy, h->st);
    CK(cudaGetLastError());
    return IFMM_OK;
}

// y = A~ x with the double-float copies of the operators on the FP32 pipe; x and y FP64 (the inner
// Krylov products of IFMM_MIXED_SOLVE)
ifmm_status matvec_dfl_impl(ifmm_handle* h, const double* x, int64_t ldx, double* y, int64_t ldy, int nrhs) {
    const int kap = h->depth, r0 = h->r0;
    void* pxt = nullptr;
    void* pout = nullptr;
    CKS(workspace(h, 90, sizeof(dfl) * (size_t)h->N * nrhs, &pxt));
    CKS(workspace(h, 91, sizeof(dfl) * (size_t)h->N * nrhs, &pout));
    dfl* xt = (dfl*)pxt;
    dfl* out = (dfl*)pout;
    std::vector<dfl*> ym(kap + 1, nullptr), zm(kap + 1, nullptr);
    for (int k = 2; k <= kap; ++k) {
        size_t len = sizeof(dfl) * ((size_t)1 << (h->dim * k)) * r0 * nrhs;
        void* a = nullptr;
        void* b = nullptr;
        CKS(workspace(h, 150 + 2 * k, len, &a));
        CKS(workspace(h, 151 + 2 * k, len, &b));
        ym[k] = (dfl*)a;
        zm[k] = (dfl*)b;
    }
    launch_mv_permute_in<dfl>(x, ldx, h->N, nrhs, h->d_perm, xt, h->st);
    launch_mv_leaf_up<dfl>(h->dim, kap, h->ops[kap].d_W0_2, h->d_leaf_start, h->d_leaf_count, r0, xt, ym[kap], nrhs, h->st);
    for (int k = kap - 1; k >= 2; --k) launch_mv_up<dfl>(h->dim, k, h->ops[k].d_W0_2, r0, ym[k + 1], ym[k], nrhs, h->st);
    for (int k = 2; k <= kap; ++k) launch_mv_m2l<dfl>(h->dim, k, h->ops[k].d_far0_2, r0, ym[k], zm[k], nrhs, h->st);
    for (int k = 2; k < kap; ++k) launch_mv_down<dfl>(h->dim, k, h->ops[k].d_W0_2, r0, zm[k], zm[k + 1], nrhs, h->st);
    launch_mv_leaf_down<dfl>(h->dim, kap, h->ops[kap].d_W0_2, h->d_leaf_start, h->d_leaf_count, r0, zm[kap], xt,
                             h->d_p2p_off, h->d_p2p2, out, nrhs, h->st);
    launch_mv_permute_out<dfl>(out, h->N, nrhs, h->d_perm, y, ldy, h->st);
    CK(cudaGetLastError());
    return IFMM_OK;
}

// FP64 GMRES(m) on A~ x = b, left-preconditioned by the IFMM solve M^{-1} (working precision T):
// every column runs its own Arnoldi process, all columns in lockstep; classical Gram-Schmidt
// applied twice; Givens rotations and the small triangular solves on the host. The monitored
// quantity |g_{j+1}| = ||M^{-1}(b - A~ x_j)|| estimates the error of x_j since M^{-1} ~ A~^{-1}.
// With IFMM_MIXED_SOLVE the preconditioner is the double-float replay and the Arnoldi products use
// the double-float matvec (both on the FP32 pipe), and a cycle ends once its estimate has fallen
// by refine_inner (or after m steps): the restart recomputes b - A~ x, so the double-float
// rounding limits each cycle's reduction, not the final accuracy (iterative refinement with a
// mixed-precision inner GMRES). In every mode only an estimate taken on a freshly computed FP64
// residual ends the solve: the recurrence's own estimate |g_{j+1}| drifts from the true
// preconditioned residual on ill-conditioned systems (measured 30x optimistic on a clustered
// cloud), so reaching refine_tol inside a cycle triggers a restart that checks it in FP64. A restart
// after a cycle that ended on refine_inner only seeds the next cycle; with IFMM_MIXED_SOLVE it
// takes the residual with the double-float matvec (rounding 2^-48 relative, far below the 0.1-0.4
// accuracy of the preconditioner it feeds), and should that residual already meet refine_tol the
// next restart recomputes it in FP64 before the solve may end.

template <typename T>
ifmm_status gmres_impl(ifmm_handle* h, const double* b, double* x, int nrhs, int64_t ld) {
    const bool inner32 = h->prm.precision == IFMM_MIXED_SOLVE;
    const double inner_red = h->prm.refine_inner > 0.0 ? h->prm.refine_inner : 1e-4;
    const int64_t N = h->N;
    const int m = std::max(1, h->prm.refine_restart);
    const double tol = h->prm.refine_tol;
    const size_t vec = (size_t)N * nrhs;
    void *pV = nullptr, *pu = nullptr, *pr = nullptr, *pd = nullptr;
    CKS(workspace(h, 60, sizeof(double) * vec * (m + 1), &pV));
    CKS(workspace(h, 61, sizeof(double) * vec, &pu));
    CKS(workspace(h, 62, sizeof(double) * vec, &pr));
    CKS(workspace(h, 63, sizeof(double) * (size_t)(m + 2) * nrhs * 2, &pd));
    void* pp = nullptr;   // per-block partial sums of the reductions (summed in a fixed order)
    CKS(workspace(h, 64, sizeof(double) * reduction_scratch_doubles(N, nrhs, m + 1), &pp));
    double* part = (double*)pp;
    double* V = (double*)pV;
    double* u = (double*)pu;
    double* r = (double*)pr;
    double* dv = (double*)pd;                 // device scratch: dots / norms / scales
    std::vector<double> H((size_t)(m + 1) * m * nrhs, 0.0), cs((size_t)m * nrhs), sn((size_t)m * nrhs),
        g((size_t)(m + 1) * nrhs), xn(nrhs, 0.0), hv((size_t)(m + 1) * nrhs), sc(nrhs);
    auto Hat = [&](int i, int j, int c) -> double& { return H[((size_t)i * m + j) * nrhs + c]; };
    for (int c = 0; c < nrhs; ++c) CK(cudaMemsetAsync(x + c * ld, 0, sizeof(double) * N, h->st));
    int it = 0;
    bool first = true;
    bool res64 = true;                        // the next restart residual in FP64
    double est = 1e300;
    auto fetch = [&](int cnt) -> ifmm_status {
        CK(cudaMemcpyAsync(hv.data(), dv, sizeof(double) * (size_t)cnt * nrhs, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        return IFMM_OK;
    };
    for (;;) {
        // z = M^{-1} (b - A~ x); fresh64: the residual is exact (x = 0) or an FP64 product
        const bool fresh64 = first || !inner32 || res64;
        if (first) {
            CKS(solve_once<T>(h, b, ld, V, N, nrhs));
        } else {
            if (fresh64) CKS(matvec_impl(h, x, ld, u, N, nrhs));
            else CKS(matvec_dfl_impl(h, x, ld, u, N, nrhs));
            CK(cudaMemsetAsync(dv, 0, sizeof(double) * 2 * nrhs, h->st));
            launch_residual(b, u, r, N, nrhs, ld, dv, part, h->st);
            CKS(solve_once<T>(h, r, N, V, N, nrhs));
        }
        CK(cudaMemsetAsync(dv, 0, sizeof(double) * nrhs, h->st));
        launch_colnorm2(V, N, N, nrhs, dv, part, h->st);
        CKS(fetch(1));
        est = 0.0;
        for (int c = 0; c < nrhs; ++c) {
            double beta = std::sqrt(hv[c]);
            if (first) xn[c] = beta;
            g[c] = beta;
            for (int i = 1; i <= m; ++i) g[(size_t)i * nrhs + c] = 0.0;
            sc[c] = beta > 0.0 ? 1.0 / beta : 0.0;
            est = std::max(est, xn[c] > 0.0 ? beta / xn[c] : 0.0);
        }
        first = false;
        if (it >= h->prm.refine_maxit) break;
        if (est <= tol) {
            if (fresh64) break;
            res64 = true;                     // confirm on an FP64 residual before ending
            continue;
        }
        const double est_cycle = est;
        CK(cudaMemcpyAsync(dv, sc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, h->st));
        launch_colscale(V, N, N, nrhs, dv, h->st);
        std::fill(H.begin(), H.end(), 0.0);
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double* Vj = V + (size_t)j * vec;
            double* Vn = V + (size_t)(j + 1) * vec;
            if (inner32) CKS(matvec_dfl_impl(h, Vj, N, u, N, nrhs));
            else CKS(matvec_impl(h, Vj, N, u, N, nrhs));
            CKS(solve_once<T>(h, u, N, Vn, N, nrhs));
            for (int pass = 0; pass < 2; ++pass) {
                CK(cudaMemsetAsync(dv, 0, sizeof(double) * (size_t)(j + 1) * nrhs, h->st));
                launch_krylov_dots(V, j + 1, Vn, N, nrhs, dv, part, h->st);
                CKS(fetch(j + 1));
                for (int i = 0; i <= j; ++i)
                    for (int c = 0; c < nrhs; ++c) {
                        Hat(i, j, c) += hv[(size_t)i * nrhs + c];
                        hv[(size_t)i * nrhs + c] = -hv[(size_t)i * nrhs + c];
                    }
                CK(cudaMemcpyAsync(dv, hv.data(), sizeof(double) * (size_t)(j + 1) * nrhs, cudaMemcpyHostToDevice, h->st));
                launch_krylov_lincomb(V, j + 1, dv, Vn, N, N, nrhs, h->st);
            }
            CK(cudaMemsetAsync(dv, 0, sizeof(double) * nrhs, h->st));
            launch_colnorm2(Vn, N, N, nrhs, dv, part, h->st);
            CKS(fetch(1));
            est = 0.0;
            for (int c = 0; c < nrhs; ++c) {
                double hn = std::sqrt(hv[c]);
                sc[c] = hn > 0.0 ? 1.0 / hn : 0.0;
                // previous rotations on column j, then a new one zeroing H(j+1, j)
                for (int i = 0; i < j; ++i) {
                    double a = Hat(i, j, c), bb = Hat(i + 1, j, c);
                    Hat(i, j, c) = cs[(size_t)i * nrhs + c] * a + sn[(size_t)i * nrhs + c] * bb;
                    Hat(i + 1, j, c) = -sn[(size_t)i * nrhs + c] * a + cs[(size_t)i * nrhs + c] * bb;
                }
                double a = Hat(j, j, c);
                double den = std::hypot(a, hn);
                double cc = den > 0.0 ? a / den : 1.0, ss = den > 0.0 ? hn / den : 0.0;
                cs[(size_t)j * nrhs + c] = cc;
                sn[(size_t)j * nrhs + c] = ss;
                Hat(j, j, c) = den;
                double gj = g[(size_t)j * nrhs + c];
                g[(size_t)(j + 1) * nrhs + c] = -ss * gj;
                g[(size_t)j * nrhs + c] = cc * gj;
                est = std::max(est, xn[c] > 0.0 ? std::fabs(g[(size_t)(j + 1) * nrhs + c]) / xn[c] : 0.0);
            }
            CK(cudaMemcpyAsync(dv, sc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, h->st));
            launch_colscale(Vn, N, N, nrhs, dv, h->st);
            ++it;
            k = j + 1;
            res64 = est <= tol;               // this cycle's restart may end the solve
            if (est <= tol || it >= h->prm.refine_maxit) break;
            if (inner32 && est <= inner_red * est_cycle) break;
        }
        // y = R^{-1} g per column, x += V y
        std::vector<double> y((size_t)k * nrhs, 0.0);
        for (int c = 0; c < nrhs; ++c)
            for (int i = k - 1; i >= 0; --i) {
                double acc = g[(size_t)i * nrhs + c];
                for (int l = i + 1; l < k; ++l) acc -= Hat(i, l, c) * y[(size_t)l * nrhs + c];
                double d = Hat(i, i, c);
                y[(size_t)i * nrhs + c] = d != 0.0 ? acc / d : 0.0;
            }
        CK(cudaMemcpyAsync(dv, y.data(), sizeof(double) * (size_t)k * nrhs, cudaMemcpyHostToDevice, h->st));
        launch_krylov_lincomb(V, k, dv, x, ld, N, nrhs, h->st);
        CK(cudaMemsetAsync(dv, 0, sizeof(double) * nrhs, h->st));
        launch_colnorm2(x, ld, N, nrhs, dv, part, h->st);
        CKS(fetch(1));
        for (int c = 0; c < nrhs; ++c) xn[c] = std::sqrt(hv[c]);
        if (it >= h->prm.refine_maxit) break;
    }
    h->stats.refine_iters = it;
    h->stats.last_update = est;
    if (est > tol) {
        h->err = "GMRES refinement stopped at refine_maxit with error estimate " + std::to_string(est);
        return IFMM_ERR_NOCONV;
    }
    return IFMM_OK;
}

template <typename T>
ifmm_status solve_impl(ifmm_handle* h, const double* b, double* x, int nrhs, int64_t ld) {
    const int64_t N = h->N;
    if (h->prm.refine_tol > 0.0 && h->prm.refine_restart > 0) return gmres_impl<T>(h, b, x, nrhs, ld);
    if (!(h->prm.refine_tol > 0.0)) {
        CKS(solve_once<T>(h, b, ld, x, ld, nrhs));
        h->stats.refine_iters = 1;
        return IFMM_OK;
    }
    void *pr = nullptr, *pd = nullptr, *pa = nullptr, *pn = nullptr;
    CKS(workspace(h, 30, sizeof(double) * (size_t)N * nrhs, &pr));
    CKS(workspace(h, 31, sizeof(double) * (size_t)N * nrhs, &pd));
    CKS(workspace(h, 32, sizeof(double) * (size_t)N * nrhs, &pa));
    CKS(workspace(h, 33, sizeof(double) * 2 * (size_t)nrhs, &pn));
    void* pp = nullptr;   // per-block partial sums of the norms (summed in a fixed order)
    CKS(workspace(h, 64, sizeof(double) * reduction_scratch_doubles(N, nrhs, 1), &pp));
    double* part = (double*)pp;
    double* r = (double*)pr;
    double* d = (double*)pd;
    double* ax = (double*)pa;
    double* nrm = (double*)pn;
    std::vector<double> hn(2 * (size_t)nrhs);
    for (int j = 0; j < nrhs; ++j) CK(cudaMemsetAsync(x + j * ld, 0, sizeof(double) * (size_t)N, h->st));
    const double* rhs = b;
    int64_t ldr = ld;
    int it = 0;
    double upd = 0.0;
    for (;;) {
        CKS(solve_once<T>(h, rhs, ldr, d, N, nrhs));
        CK(cudaMemsetAsync(nrm, 0, sizeof(double) * 2 * nrhs, h->st));
        launch_axpy_norms(x, d, N, nrhs, ld, nrm, part, h->st);
        CK(cudaMemcpyAsync(hn.data(), nrm, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        ++it;
        upd = 0.0;
        for (int j = 0; j < nrhs; ++j) upd = std::max(upd, std::sqrt(hn[2 * j] / std::max(hn[2 * j + 1], 1e-300)));
        if (upd <= h->prm.refine_tol || it >= h->prm.refine_maxit) break;
        CKS(matvec_impl(h, x, ld, ax, N, nrhs));
        CK(cudaMemsetAsync(nrm, 0, sizeof(double) * 2 * nrhs, h->st));
        launch_residual(b, ax, r, N, nrhs, ld, nrm, part, h->st);
        CK(cudaMemcpyAsync(hn.data(), nrm, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        double res = 0.0;
        for (int j = 0; j < nrhs; ++j) res = std::max(res, std::sqrt(hn[2 * j] / std::max(hn[2 * j + 1], 1e-300)));
        h->stats.last_residual = res;
        rhs = r;
        ldr = N;
    }
    h->stats.refine_iters = it;
    h->stats.last_update = upd;
    if (upd > h->prm.refine_tol) {
        h->err = "iterative refinement stopped at refine_maxit with update " + std::to_string(upd);
        return IFMM_ERR_NOCONV;
    }
    return IFMM_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
// Batched calls: a native scheduler runs independent systems concurrently. Systems are taken in
// order of decreasing work (N x nrhs) and each goes to the worker with the least work so far
// (longest-processing-time-first); a worker runs its systems in that order on their own streams.
namespace {
template <class F>
ifmm_status run_batch(ifmm_h* hs, int n, int workers, const std::vector<double>& work, ifmm_status* status_out,
                      F one) {
    if (!hs || n <= 0) return IFMM_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!hs[i]) return IFMM_ERR_INVALID_ARG;
    if (workers <= 0) workers = std::min(n, 16);
    workers = std::min(workers, n);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<std::vector<int>> lists(workers);
    std::vector<double> load(workers, 0.0);
    for (int i : order) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[w].push_back(i);
        load[w] += work[i];
    }
    std::vector<ifmm_status> st(n, IFMM_OK);
    std::vector<std::thread> pool;
    for (int w = 0; w < workers; ++w)
        pool.emplace_back([&, w]() {
            for (int i : lists[w]) {
                cudaSetDevice(hs[i]->device);
                st[i] = one(i);
            }
        });
    for (auto& t : pool) t.join();
    ifmm_status first = IFMM_OK;
    for (int i = 0; i < n; ++i) {
        if (status_out) status_out[i] = st[i];
        if (first == IFMM_OK && st[i] != IFMM_OK) first = st[i];
    }
    return first;
}
}  // namespace


extern "C" {

void ifmm_default_params(ifmm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dim = 2;
    p->depth = 3;
    p->cheb_p = 4;
    p->r_cap = 0;
    p->eps = 1e-10;
    p->diag = 1.0;
    p->box[0] = 0.0; p->box[1] = 0.0; p->box[2] = 1.0;
    p->precision = IFMM_FP64;
    p->tau_ref = 1;
    p->refine_tol = 0.0;
    p->refine_maxit = 100;
    p->refine_restart = 60;
    p->refine_inner = 1e-4;
    p->leaf_max = 64;
    p->tc_products = 0;
    p->svd_eps = 0.0;
    p->z0 = 0.0;
}

// Smallest depth 2..10 of the uniform tree whose fullest leaf holds at most leaf_max points, with the
// build's leaf rule (floor of the box-relative coordinate times 2^depth, the upper edge clamped into
// the last box); 10 if none. Host only.
int ifmm_auto_depth(const double* pts_host, int64_t N, const double* box, int leaf_max) {
    if (!pts_host || N <= 0 || leaf_max <= 0) return -1;
    double x0 = 0.0, y0 = 0.0, L = 1.0;
    if (box && box[2] > 0.0) { x0 = box[0]; y0 = box[1]; L = box[2]; }
    for (int depth = 2; depth <= 10; ++depth) {
        const int side = 1 << depth;
        std::vector<int> cnt((size_t)side * side, 0);
        int mx = 0;
        for (int64_t t = 0; t < N; ++t) {
            const double ux = std::fmin(std::fmax((pts_host[2 * t] - x0) / L, 0.0), 1.0);
            const double uy = std::fmin(std::fmax((pts_host[2 * t + 1] - y0) / L, 0.0), 1.0);
            const int ix = std::min((int)std::floor(ux * side), side - 1);
            const int iy = std::min((int)std::floor(uy * side), side - 1);
            mx = std::max(mx, ++cnt[(size_t)iy * side + ix]);
        }
        if (mx <= leaf_max) return depth;
    }
    return 10;
}

ifmm_status ifmm_build(const double* pts_host, int64_t N, int kernel, const ifmm_params* p, void* stream,
                       ifmm_h* out) {
    if (out) *out = nullptr;
    if (!pts_host || !p || !out || N <= 0 || N >= (1ll << 31)) return IFMM_ERR_INVALID_ARG;
    if ((p->dim != 2 && p->dim != 3) || (p->depth != 0 && (p->depth < 2 || p->depth > 10)) || p->cheb_p < 1 ||
        p->cheb_p > 8)
        return IFMM_ERR_INVALID_ARG;
    if (p->depth == 0 && p->leaf_max <= 0) return IFMM_ERR_INVALID_ARG;
    // octree: p^3 <= 64 Chebyshev nodes (the QR of the bases keeps 64 columns in shared memory),
    // an explicit depth <= 6, the double-float or FP64 products (the tensor-core replay keeps the
    // quadtree's 8 neighbour panels per box)
    if (p->dim == 3 && (p->cheb_p > 4 || p->depth == 0 || p->depth > 6 || p->tc_products != 0))
        return IFMM_ERR_INVALID_ARG;
    if (!std::isfinite(p->z0)) return IFMM_ERR_INVALID_ARG;
    if (kernel < IFMM_K_INV_R || kernel > IFMM_K_R2LOG_REG) return IFMM_ERR_INVALID_ARG;
    if (kernel != IFMM_K_INV_R && !(p->kparam[0] > 0.0)) return IFMM_ERR_INVALID_ARG;
    if (!(p->eps >= 0.0) || !std::isfinite(p->diag)) return IFMM_ERR_INVALID_ARG;
    if (p->precision != IFMM_FP64 && p->precision != IFMM_MIXED && p->precision != IFMM_MIXED_SOLVE)
        return IFMM_ERR_INVALID_ARG;
    if (p->tau_ref < 0 || p->tau_ref > 2) return IFMM_ERR_INVALID_ARG;
    if (p->r_cap > 0 && p->r_cap < p->cheb_p * p->cheb_p) return IFMM_ERR_INVALID_ARG;
    if (p->tc_products < 0 || p->tc_products > 2) return IFMM_ERR_INVALID_ARG;
    if (!(p->svd_eps >= 0.0 && p->svd_eps < 1.0)) return IFMM_ERR_INVALID_ARG;
    for (int64_t i = 0; i < (int64_t)p->dim * N; ++i)
        if (!std::isfinite(pts_host[i])) return IFMM_ERR_INVALID_ARG;
    ifmm_handle* h = new ifmm_handle();
    h->prm = *p;
    if (!(h->prm.box[2] > 0.0)) { h->prm.box[0] = 0.0; h->prm.box[1] = 0.0; h->prm.box[2] = 1.0; h->prm.z0 = 0.0; }
    if (h->prm.refine_maxit <= 0) h->prm.refine_maxit = 100;
    if (h->prm.refine_restart < 0 || h->prm.refine_restart > 200) {
        delete h;
        return IFMM_ERR_INVALID_ARG;
    }
    h->kernel = kernel;
    h->N = N;
    if (h->prm.depth == 0) h->prm.depth = ifmm_auto_depth(pts_host, N, h->prm.box, h->prm.leaf_max);
    h->depth = h->prm.depth;
    cudaGetDevice(&h->device);
    h->pool = library_pool(h->device);
    h->p = p->cheb_p;
    h->dim = p->dim;
    h->r0 = p->dim == 3 ? p->cheb_p * p->cheb_p * p->cheb_p : p->cheb_p * p->cheb_p;
    h->st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    ifmm_status s = do_build(h, pts_host);
    if (s != IFMM_OK) {
        ifmm_destroy(h);
        return s;
    }
    h->stats.t_build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h->stats.n_points = N;
    h->stats.depth = h->depth;
    *out = h;
    return IFMM_OK;
}

ifmm_status ifmm_factor(ifmm_h h) {
    if (!h) return IFMM_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    h->err.clear();
    release_factors(h);
    auto t0 = std::chrono::steady_clock::now();
    ifmm_status s = h->prm.precision == IFMM_MIXED ? factor_impl<float>(h) : factor_impl<double>(h);
    // the double-float replay reads double-float copies of the factors; the tensor-core replay
    // reads digit slabs of the FP64 factors
    if ((s == IFMM_OK || s == IFMM_ERR_RANK_OVERFLOW) && h->prm.precision == IFMM_MIXED_SOLVE && h->prm.tc_products) {
        ifmm_status s2 = presplit_factors(h);
        if (s2 != IFMM_OK) {
            h->factored = false;
            return s2;
        }
    }
    if ((s == IFMM_OK || s == IFMM_ERR_RANK_OVERFLOW) && h->prm.precision == IFMM_MIXED_SOLVE && !h->prm.tc_products) {
        ifmm_status s2 = split_factors(h);
        if (s2 != IFMM_OK) {
            h->factored = false;
            return s2;
        }
    }
    h->stats.t_factor_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (s != IFMM_OK && s != IFMM_ERR_RANK_OVERFLOW) h->factored = false;
    return s;
}

ifmm_status ifmm_solve(ifmm_h h, const double* b_dev, double* x_dev, int nrhs, int64_t ld) {
    if (!h || !b_dev || !x_dev || nrhs < 1 || nrhs > 1024 || ld < h->N) return IFMM_ERR_INVALID_ARG;
    if (!h->factored) {
        h->err = "ifmm_solve before ifmm_factor";
        return IFMM_ERR_STATE;
    }
    DeviceGuard dg(h->device);
    h->err.clear();
    auto t0 = std::chrono::steady_clock::now();
    const long long l0 = launches_so_far();
    // IFMM_MIXED_SOLVE replays in double-float on the FP32 pipe, or with FP64 vectors and the replay
    // products on the tensor cores (tc_products)
    const bool dfl_replay = h->prm.precision == IFMM_MIXED_SOLVE && !h->prm.tc_products;
    ifmm_status s = h->prm.precision == IFMM_MIXED ? solve_impl<float>(h, b_dev, x_dev, nrhs, ld)
                    : dfl_replay                   ? solve_impl<dfl>(h, b_dev, x_dev, nrhs, ld)
                                                   : solve_impl<double>(h, b_dev, x_dev, nrhs, ld);
    h->stats.launches_solve = launches_so_far() - l0;
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (s == IFMM_OK && e != cudaSuccess) {
        h->err = std::string("solve: ") + cudaGetErrorString(e);
        s = IFMM_ERR_CUDA;
    }
    h->stats.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return s;
}

// Transposed solve. Every kernel of the library is symmetric, K(x, y) = K(y, x), and the build
// keeps A~ symmetric: P2P_ji = P2P_ij^T, M2L_ji = M2L_ij^T, L2P = P2M^T; the elimination compresses
// the fill of every box with one basis for its row and its column (F_qp = F_pq^T), so the compressed
// matrix that the factors invert is symmetric as well. A~^T x = b is therefore the system of
// ifmm_solve, solved by the same replay of the factors.
ifmm_status ifmm_solve_T(ifmm_h h, const double* b_dev, double* x_dev, int nrhs, int64_t ld) {
    if (!h) return IFMM_ERR_INVALID_ARG;
    if (h->kernel < IFMM_K_INV_R || h->kernel > IFMM_K_R2LOG_REG) {
        h->err = "ifmm_solve_T: the transposed replay is only provided for symmetric kernels";
        return IFMM_ERR_INVALID_ARG;
    }
    return ifmm_solve(h, b_dev, x_dev, nrhs, ld);
}

ifmm_status ifmm_factor_batch(ifmm_h* hs, int n, int workers, ifmm_status* status_out) {
    if (!hs || n <= 0) return IFMM_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!hs[i]) return IFMM_ERR_INVALID_ARG;
    // one device and one precision: the systems' levels run in lockstep, each colour one launch per
    // kernel over all of them
    bool fused = true;
    for (int i = 1; i < n; ++i)
        fused = fused && hs[i]->device == hs[0]->device && hs[i]->prm.precision == hs[0]->prm.precision &&
                hs[i]->prm.tc_products == hs[0]->prm.tc_products && hs[i]->dim == hs[0]->dim;
    if (fused) {
        DeviceGuard dg(hs[0]->device);
        if (workers <= 0) workers = std::min(n, 16);
        auto t0 = std::chrono::steady_clock::now();
        std::vector<ifmm_status> st(n, IFMM_OK);
        ifmm_status s = hs[0]->prm.precision == IFMM_MIXED ? factor_fused<float>(hs, n, workers, st.data())
                                                           : factor_fused<double>(hs, n, workers, st.data());
        (void)s;
        // the solve's copies of the factors (IFMM_MIXED_SOLVE), per system
        std::vector<int> idx;
        for (int i = 0; i < n; ++i)
            if ((st[i] == IFMM_OK || st[i] == IFMM_ERR_RANK_OVERFLOW) && hs[i]->prm.precision == IFMM_MIXED_SOLVE)
                idx.push_back(i);
        const int dev = hs[0]->device;
        for_each_system(idx, workers, [&](int i) {
            cudaSetDevice(dev);
            ifmm_status s2 = hs[i]->prm.tc_products ? presplit_factors(hs[i]) : split_factors(hs[i]);
            if (s2 == IFMM_OK) s2 = cudaStreamSynchronize(hs[i]->st) == cudaSuccess ? IFMM_OK : IFMM_ERR_CUDA;
            if (s2 != IFMM_OK) {
                hs[i]->factored = false;
                st[i] = s2;
            }
        });
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        ifmm_status first = IFMM_OK;
        for (int i = 0; i < n; ++i) {
            hs[i]->stats.t_factor_ms = ms;   // the whole batch's time
            if (status_out) status_out[i] = st[i];
            if (first == IFMM_OK && st[i] != IFMM_OK) first = st[i];
        }
        return first;
    }
    std::vector<double> work(n);
    for (int i = 0; i < n; ++i) work[i] = hs[i] ? (double)hs[i]->N : 0.0;
    return run_batch(hs, n, workers, work, status_out, [&](int i) {
        hs[i]->in_batch = true;
        const ifmm_status s = ifmm_factor(hs[i]);
        hs[i]->in_batch = false;
        return s;
    });
}

// Autotuner of the batched launches (no counterpart in the paper): times the panel and Schur
// launches of ifmm_factor_batch on the given systems for each candidate split and keeps, per
// bucket of (kernel, double-float products, ceil(log2 nmax), ceil(log2 boxes)), the fastest.
ifmm_status ifmm_autotune(ifmm_h* hs, int n, int workers) {
    if (!hs || n <= 0) return IFMM_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!hs[i]) return IFMM_ERR_INVALID_ARG;
    DeviceGuard dg(hs[0]->device);
    static const int cand[5] = {1, 2, 4, 8, 16};
    // warm-up: one-time kernel set-up out of the measured runs
    ifmm_status s = ifmm_factor_batch(hs, n, workers, nullptr);
    if (s != IFMM_OK && s != IFMM_ERR_RANK_OVERFLOW) return s;
    auto table = tune_table_get();
    for (int kernel = 0; kernel < 2; ++kernel) {
        std::map<std::tuple<int, int, int, int>, std::vector<double>> times;
        for (int c = 0; c < 5; ++c) {
            tune_set_force(kernel == 0 ? cand[c] : 0, kernel == 1 ? cand[c] : 0);
            tune_record(true);
            s = ifmm_factor_batch(hs, n, workers, nullptr);
            cudaDeviceSynchronize();
            tune_record(false);
            auto m = tune_collect(kernel);
            if (s != IFMM_OK && s != IFMM_ERR_RANK_OVERFLOW) {
                tune_set_force(0, 0);
                return s;
            }
            for (auto& kv : m) {
                auto& v = times[kv.first];
                v.resize(5, 1e300);
                v[c] = kv.second;
            }
        }
        for (auto& kv : times) {
            int bc = 0;
            for (int c = 1; c < 5; ++c)
                if (kv.second[c] < kv.second[bc]) bc = c;
            table[kv.first] = cand[bc];
        }
    }
    tune_set_force(0, 0);
    tune_table_set(table);
    return ifmm_factor_batch(hs, n, workers, nullptr);   // leave the systems factored with the table
}

ifmm_status ifmm_autotune_save(const char* path) {
    if (!path) return IFMM_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "w");
    if (!f) return IFMM_ERR_INVALID_ARG;
    std::fprintf(f, "# ifmm autotune table: kernel (0 panel, 1 Schur), double-float products (0/1), "
                    "ceil(log2 nmax), ceil(log2 boxes of the launch), split\n");
    for (auto& kv : tune_table_get())
        std::fprintf(f, "%d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                     std::get<3>(kv.first), kv.second);
    const bool ok = std::fclose(f) == 0;
    return ok ? IFMM_OK : IFMM_ERR_INVALID_ARG;
}

ifmm_status ifmm_autotune_load(const char* path) {
    if (!path) return IFMM_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "r");
    if (!f) return IFMM_ERR_INVALID_ARG;
    std::map<std::tuple<int, int, int, int>, int> t;
    char line[512];
    bool ok = true;
    while (std::fgets(line, sizeof(line), f)) {
        const char* c = line;
        while (*c == ' ' || *c == '\t') ++c;
        if (*c == '#' || *c == '\n' || *c == '\r' || *c == 0) continue;
        int k, df, lb, bb, z;
        char extra = 0;
        if (std::sscanf(c, "%d %d %d %d %d %c", &k, &df, &lb, &bb, &z, &extra) != 5 || k < 0 || k > 1 || df < 0 ||
            df > 1 || lb < 0 || lb > 30 || bb < 0 || bb > 30 || z < 1 || z > 64) {
            ok = false;
            break;
        }
        t[std::make_tuple(k, df, lb, bb)] = z;
    }
    std::fclose(f);
    if (!ok) return IFMM_ERR_INVALID_ARG;
    tune_table_set(t);
    return IFMM_OK;
}

void ifmm_autotune_clear(void) { tune_table_set({}); }

int ifmm_autotune_size(void) { return (int)tune_table_get().size(); }

ifmm_status ifmm_set_compress_cluster(int max_blocks) {
    return set_compress_cluster(max_blocks) == 0 ? IFMM_OK : IFMM_ERR_INVALID_ARG;
}

ifmm_status ifmm_solve_batch(ifmm_h* hs, int n, const double* const* b_dev, double* const* x_dev, const int* nrhs,
                             const int64_t* ld, int workers, ifmm_status* status_out) {
    if (!hs || n <= 0 || !b_dev || !x_dev || !nrhs || !ld) return IFMM_ERR_INVALID_ARG;
    std::vector<double> work(n);
    for (int i = 0; i < n; ++i) work[i] = hs[i] ? (double)hs[i]->N * std::max(nrhs[i], 1) : 0.0;
    return run_batch(hs, n, workers, work, status_out,
                     [&](int i) { return ifmm_solve(hs[i], b_dev[i], x_dev[i], nrhs[i], ld[i]); });
}

ifmm_status ifmm_solve_host(ifmm_h h, const double* b_host, double* x_host, int nrhs, int64_t ld) {
    if (!h || !b_host || !x_host || nrhs < 1 || nrhs > 1024 || ld < h->N) return IFMM_ERR_INVALID_ARG;
    if (!h->factored) {
        h->err = "ifmm_solve_host before ifmm_factor";
        return IFMM_ERR_STATE;
    }
    DeviceGuard dg(h->device);
    void *pb = nullptr, *px = nullptr;
    CKS(workspace(h, 80, sizeof(double) * (size_t)h->N * nrhs, &pb));
    CKS(workspace(h, 81, sizeof(double) * (size_t)h->N * nrhs, &px));
    // one copy per column, or one for the whole block when the columns are contiguous (ld = N);
    // from page-locked host memory the copies run at the link's rate, from pageable memory the
    // driver stages them
    const int ncopy = ld == h->N ? 1 : nrhs;
    const size_t cbytes = sizeof(double) * h->N * (ld == h->N ? (size_t)nrhs : 1);
    for (int j = 0; j < ncopy; ++j)
        CK(cudaMemcpyAsync((double*)pb + (size_t)j * h->N, b_host + (size_t)j * ld, cbytes, cudaMemcpyHostToDevice,
                           h->st));
    ifmm_status s = ifmm_solve(h, (double*)pb, (double*)px, nrhs, h->N);
    if (s != IFMM_OK && s != IFMM_ERR_NOCONV) return s;
    for (int j = 0; j < ncopy; ++j)
        CK(cudaMemcpyAsync(x_host + (size_t)j * ld, (double*)px + (size_t)j * h->N, cbytes, cudaMemcpyDeviceToHost,
                           h->st));
    CK(cudaStreamSynchronize(h->st));
    return s;
}

ifmm_status ifmm_matvec(ifmm_h h, const double* x_dev, double* y_dev, int nrhs, int64_t ld) {
    if (!h || !x_dev || !y_dev || nrhs < 1 || nrhs > 1024 || ld < h->N) return IFMM_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    h->err.clear();
    CKS(matvec_impl(h, x_dev, ld, y_dev, ld, nrhs));
    CK(cudaStreamSynchronize(h->st));
    return IFMM_OK;
}

ifmm_status ifmm_get_ranks(ifmm_h h, int level, int* out_host) {
    if (!h || !out_host || level < 2 || level > h->depth) return IFMM_ERR_INVALID_ARG;
    if (!h->factored) return IFMM_ERR_STATE;
    const FLevel& L = h->lv[level];
    std::copy(L.r.begin(), L.r.end(), out_host);
    return IFMM_OK;
}

ifmm_status ifmm_get_stats(ifmm_h h, ifmm_stats* s) {
    if (!h || !s) return IFMM_ERR_INVALID_ARG;
    h->stats.device_bytes = h->bytes;
    *s = h->stats;
    return IFMM_OK;
}

const char* ifmm_last_error(ifmm_h h) { return h ? h->err.c_str() : "null handle"; }

void ifmm_destroy(ifmm_h h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    for (auto& a : h->allocs) {
        if (h->pool) cudaFreeAsync(a.first, h->st);
        else cudaFree(a.first);
    }
    if (h->pool) {
        if (h->st) cudaStreamSynchronize(h->st);
        else cudaDeviceSynchronize();
        cudaMemPoolTrimTo(h->pool, 0);
    }
    delete h;
}

// ------------------------------------------------------------------------------------------------
// FMM matvec without any device allocation
// ------------------------------------------------------------------------------------------------
}  // extern "C"

namespace {

// Scratch of ifmm_matvec_noalloc: a fixed 32 MiB array in the library's device image. Every GPU
// that loads the library holds it until the process exits; all calls share it.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {nullptr};   // device address of g_noalloc_scratch, per device ordinal

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" ifmm_status ifmm_matvec_noalloc(ifmm_h h, const double* x_dev, double* y_dev, int nrhs, int64_t ld) {
    if (!h || !x_dev || !y_dev || nrhs < 1 || nrhs > 1024 || ld < h->N) return IFMM_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);   // the handle's device is current from here on
    h->err.clear();
    const int kap = h->depth, r0 = h->r0;
    // carve the scratch: tree-order input and output, then multipoles and locals per level
    const size_t vec = align256(sizeof(double) * (size_t)h->N * nrhs);
    size_t need = 2 * vec;
    std::vector<size_t> lvl(kap + 1, 0);
    for (int k = 2; k <= kap; ++k) {
        lvl[k] = align256(sizeof(double) * ((size_t)1 << (h->dim * k)) * r0 * nrhs);
        need += 2 * lvl[k];
    }
    if (need > kNoAllocScratchBytes) {
        h->err = "ifmm_matvec_noalloc: this problem needs " + std::to_string(need) +
                 " bytes of scratch; the fixed limit is " + std::to_string(kNoAllocScratchBytes) +
                 " bytes (reduce N * nrhs, or use ifmm_matvec)";
        return IFMM_ERR_INVALID_ARG;
    }
    // set-up, once per device, with that device (the handle's) current: the host-side name of the
    // array is not a device address, so fetch the address the kernels must be given
    const int dev = h->device;
    if (dev < 0 || dev >= 256) {
        h->err = "ifmm_matvec_noalloc: device ordinal out of range";
        return IFMM_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                h->err = std::string("ifmm_matvec_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
                return IFMM_ERR_CUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    }
    double* xt = reinterpret_cast<double*>(base);
    double* out = reinterpret_cast<double*>(base + vec);
    std::vector<double*> ym(kap + 1, nullptr), zm(kap + 1, nullptr);
    size_t off = 2 * vec;
    for (int k = 2; k <= kap; ++k) {
        ym[k] = reinterpret_cast<double*>(base + off);
        off += lvl[k];
        zm[k] = reinterpret_cast<double*>(base + off);
        off += lvl[k];
    }
    // every scratch vector is written before it is read (the M2L launch clears the locals first)
    launch_mv_permute_in(x_dev, ld, h->N, nrhs, h->d_perm, xt, h->st);
    launch_mv_leaf_up(h->dim, kap, h->ops[kap].d_W0, h->d_leaf_start, h->d_leaf_count, r0, xt, ym[kap], nrhs, h->st);
    for (int k = kap - 1; k >= 2; --k) launch_mv_up(h->dim, k, h->ops[k].d_W0, r0, ym[k + 1], ym[k], nrhs, h->st);
    for (int k = 2; k <= kap; ++k) launch_mv_m2l(h->dim, k, h->ops[k].d_far0, r0, ym[k], zm[k], nrhs, h->st);
    for (int k = 2; k < kap; ++k) launch_mv_down(h->dim, k, h->ops[k].d_W0, r0, zm[k], zm[k + 1], nrhs, h->st);
    launch_mv_leaf_down(h->dim, kap, h->ops[kap].d_W0, h->d_leaf_start, h->d_leaf_count, r0, zm[kap], xt, h->d_p2p_off,
                        h->d_p2p, out, nrhs, h->st);
    launch_mv_permute_out(out, h->N, nrhs, h->d_perm, y_dev, ld, h->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->st));
    return IFMM_OK;
}
