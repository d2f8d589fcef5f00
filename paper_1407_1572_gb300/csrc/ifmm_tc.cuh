// ifmm_tc.cuh -- FP64-accurate products on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The dense contractions of the elimination (the Schur update C_p X_q of Algorithm 1 and its
// panel products) are real GEMMs, but GB300 has no fast FP64 tensor path. They run here as exact
// integer arithmetic on the bf16 tensor cores (the splitting idea of Ozaki et al.):
//
//  * each row i of A is scaled by 2^-a_i and each column j of B by 2^-b_j (powers of two chosen
//    from the largest exponent of the row / column, so scaled entries lie in (-1, 1)), and every
//    scaled entry is cut into S = 8 digits of 7 bits, x = sum_s d_s 2^-7(s+1) (|d_s| <= 127, all of
//    the sign of x, the remainder below 2^-56) -- the digits are small integers, exact in bf16;
//  * C_ij = 2^(a_i + b_j) sum_g 2^-7(g+2) P_g(i, j), where P_g = sum_{s+t=g} A_s B_t collects the
//    digit products of weight g. One tcgen05.mma of kind::f16 per digit pair (s, t), s + t <= 7
//    (36 pairs), accumulates into the FP32 accumulator of its weight g in tensor memory. Each digit
//    product is an integer below 2^14, and over at most 128 terms of K the eight pairs of one
//    weight stay below 8 * 128 * 127^2 < 2^24: every accumulator is an exact integer;
//  * after every 128 terms of K the accumulators are read back (tcgen05.ld), converted to integers
//    and combined in 64-bit integer arithmetic into H = floor(2^39 sum_g 2^-7g P_g) (|H| < 2^61),
//    which integer operations turn into an FP64 number scaled by 2^(a_i + b_j) (truncated to 53
//    bits); the read-backs of one output are summed in FP64.
// Dropped digits (below 2^-56 of the row's or column's largest entry) and dropped weights g >= 8
// leave about 2^-52 of |A| |B| (a bit-exact emulation on normal rows scaled over 2^+-30: 2^-52.2;
// seven digits gave 2^-45.4), better than the 2^-48 of a double-float product, and no FP64
// arithmetic is spent on the products: the FP64 pipe of GB300 (2 fused multiply-adds per SM per
// clock) would take as long as the tensor cores' whole work.
//
// Layout. Operand tiles live in shared memory in the tensor cores' canonical K-major layout
// without swizzle: 8 x 8 "core matrices" of bf16 (8 rows of 16 bytes), the core matrices of one
// 8-row group consecutive along K (leading byte offset 128 B), the 8-row groups one after another
// (stride byte offset 512 B for a 32-wide K chunk). One elected thread issues the 28 x 2 MMAs of a
// K chunk of 32 and commits them to an mbarrier; all waits are bounded and report a timeout into
// the caller's status word instead of hanging.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ifmm_internal.h"

namespace ifmm {
namespace tc {

constexpr int kSlices = 8;                 // digits per entry
constexpr int kDigitBits = 7;
constexpr int kPairs = 36;                 // digit pairs (s, t) with s + t <= 7
constexpr int kTM = 128;                   // rows of a tile (one TMEM lane per row)
constexpr int kTN = 32;                    // columns of a tile
constexpr int kKC = 32;                    // K per shared-memory chunk
constexpr int kChunksPerDrain = 4;         // 128 terms of K between accumulator read-backs
constexpr int kThreads = 128;              // four warps: one TMEM lane quarter each
constexpr int kTmemCols = 256;             // 8 accumulators x 32 columns
constexpr int kASliceBytes = kTM * kKC * 2;     // 8 KB
constexpr int kBSliceBytes = kTN * kKC * 2;     // 2 KB
// dynamic shared memory of a CTA that runs tc_gemm (1 KB aligned base)
constexpr int kSmemBytes = kSlices * (kASliceBytes + kBSliceBytes) + (kTM + kTN) * 4 + 64;

// status bit set when a bounded wait on the tensor cores ran out
constexpr int kErrTimeout = DEV_ERR_TIMEOUT;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of an R x 32 K-major tile in the canonical no-swizzle layout
__device__ __forceinline__ uint32_t core_offset(int r, int k) {
    return (uint32_t)((r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading byte offset (between core matrices
// along K), stride byte offset (between 8-row groups), fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bf16 bit pattern of the integer digit d, |d| <= 127 (exact: at most 7 significant bits). The
// float of |d| is formed as (2^23 + |d|) - 2^23 on the FP32 pipe; its high half is the bf16.
__device__ __forceinline__ uint32_t bf16_digit(uint32_t mag, uint32_t neg) {
    const float f = __fsub_rn(__uint_as_float(0x4B000000u | mag), 8388608.0f);
    return (__float_as_uint(f) >> 16) | (mag ? (neg << 15) : 0u);
}

// Biased FP64 exponent field of v (0 for zero and subnormals, which the split flushes).
__device__ __forceinline__ int exp_field(double v) {
    return (int)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF;
}

// The 8 digits of v scaled by 2^-(E - 1022), E = the largest exponent field of v's row / column:
// F = floor(|v| 2^-(E - 1022) 2^56) = M53 2^(e - E + 3) (< 2^56), d_s = (F >> (49 - 7 s)) & 127,
// packed as bf16 bit patterns into out[s].
__device__ __forceinline__ void split_digits(double v, int E, uint32_t* out) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)(b >> 52) & 0x7FF;
    const uint32_t neg = (uint32_t)(b >> 63);
    const int d = E - e;                      // >= 0
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    unsigned long long F = 0;
    if (e != 0 && d < 56) F = d <= 3 ? m << (3 - d) : m >> (d - 3);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) out[s] = bf16_digit((uint32_t)(F >> (49 - 7 * s)) & 127u, neg);
}

// ---- tcgen05 / mbarrier wrappers ------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"((uint32_t)kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"((uint32_t)kTmemCols));
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// wait for the mbarrier phase `parity` to complete; false after about 2^22 tries with back-off
// (seconds), so that a fault in the issue path cannot hang the GPU
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(256);
    }
    return false;
}
// 8 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
// 16 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// exact integer value of an integer-valued float below 2^24 in magnitude
__device__ __forceinline__ long long exact_int(uint32_t bits) { return (long long)__float2int_rn(__uint_as_float(bits)); }

// H 2^sh as an FP64 number, assembled with integer operations only (the leading bit found by a
// count of leading zeros, the significand truncated to 53 bits); results below 2^-1022 are flushed
// to zero, above the FP64 range they become infinite
__device__ __forceinline__ double scaled_int(long long H, int sh) {
    if (H == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)H & 0x8000000000000000ull;
    const unsigned long long mag = H < 0 ? (unsigned long long)(-H) : (unsigned long long)H;
    const int lz = __clzll((long long)mag);
    const unsigned long long m = mag << lz;                  // leading one at bit 63
    const int e = 63 - lz + 1023 + sh;                        // biased exponent of H 2^sh
    if (e <= 0) return 0.0;
    if (e >= 0x7FF) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
    return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | ((m >> 11) & 0xFFFFFFFFFFFFFull)));
}

// Per-CTA state of the tensor-core GEMM: shared-memory carve-up, TMEM base, mbarrier phase.
struct Ctx {
    uint8_t* a_sl;         // kSlices A slice tiles (kTM x kKC bf16 each)
    uint8_t* b_sl;         // kSlices B slice tiles (kTN x kKC bf16 each)
    int* rexp;             // [kTM] largest exponent field of each tile row of A
    int* cexp;             // [kTN] ... of each tile column of B
    uint64_t* bar;
    uint32_t* tslot;
    uint32_t tmem;
    uint32_t phase;
    int* status;
    int zng;               // row groups of the A slices that may hold data (the rest are zero)
    bool ok;
};

// Set up a CTA (all kThreads threads): carve shared memory, init the mbarrier, allocate TMEM.
__device__ __forceinline__ void ctx_init(Ctx& c, uint8_t* smem, int* status) {
    c.a_sl = smem;
    c.b_sl = smem + kSlices * kASliceBytes;
    c.rexp = reinterpret_cast<int*>(c.b_sl + kSlices * kBSliceBytes);
    c.cexp = c.rexp + kTM;
    c.bar = reinterpret_cast<uint64_t*>(c.cexp + kTN + 2);   // 8-byte aligned: offset (kTM + kTN + 2) * 4
    c.tslot = reinterpret_cast<uint32_t*>(c.bar + 1);
    c.phase = 0;
    c.status = status;
    c.zng = kTM / 8;
    c.ok = true;
    if (threadIdx.x == 0) mbar_init(c.bar);
    if ((threadIdx.x >> 5) == 0) tmem_alloc(c.tslot);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    c.tmem = *c.tslot;
}

// Release TMEM (all threads; after the last read-back).
__device__ __forceinline__ void ctx_release(Ctx& c) {
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(c.tmem);
}

// C = A B for an M x N output, K deep, in FP64 accuracy. la(i, k) / lb(k, j) return FP64 operands,
// epi(i, j, v) receives each output once. Output tiles of kTM x kTN with index tile0 (mod tstride)
// belong to this CTA. All kThreads threads call it; the Ctx is set up once per CTA.
template <class LA, class LB, class EPI>
__device__ void tc_gemm(Ctx& c, int M, int N, int K, LA la, LB lb, EPI epi, int tile0, int tstride) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tn = (N + kTN - 1) / kTN, tm = (M + kTM - 1) / kTM;
    const uint32_t idesc = instr_desc(kTM, kTN);
    for (int tile = tile0; tile < tm * tn; tile += tstride) {
        const int m0 = (tile / tn) * kTM, n0 = (tile % tn) * kTN;
        const int mm = min(kTM, M - m0), nn = min(kTN, N - n0);
        // per-tile exponents: the largest exponent field of each row of A and each column of B
        // over the whole K (a warp per row, a thread per column)
        for (int r = warp; r < kTM; r += kThreads / 32) {
            int e = 0;
            if (r < mm)
                for (int k = lane; k < K; k += 32) e = max(e, exp_field(la(m0 + r, k)));
            for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
            if (lane == 0) c.rexp[r] = e;
        }
        if (tid < kTN) {
            int e = 0;
            if (tid < nn)
                for (int k = 0; k < K; ++k) e = max(e, exp_field(lb(k, n0 + tid)));
            c.cexp[tid] = e;
        }
        __syncthreads();
        double acc[kTN];
#pragma unroll
        for (int j = 0; j < kTN; ++j) acc[j] = 0.0;
        const int er = c.rexp[tid];
        const int nchunks = (K + kKC - 1) / kKC;
        for (int ch = 0; ch < nchunks; ++ch) {
            const int k0 = ch * kKC;
            // ---- split the A chunk (kTM x kKC) and the B chunk (kTN x kKC) into digit tiles
            for (int t = tid; t < kTM * (kKC / 2); t += kThreads) {
                const int r = t / (kKC / 2), kp = (t - r * (kKC / 2)) * 2;
                uint32_t d0[kSlices], d1[kSlices];
                const int gk = k0 + kp;
                const bool live = r < mm;
                split_digits(live && gk < K ? la(m0 + r, gk) : 0.0, c.rexp[r], d0);
                split_digits(live && gk + 1 < K ? la(m0 + r, gk + 1) : 0.0, c.rexp[r], d1);
                const uint32_t off = core_offset(r, kp);
#pragma unroll
                for (int s = 0; s < kSlices; ++s)
                    *reinterpret_cast<uint32_t*>(c.a_sl + s * kASliceBytes + off) = d0[s] | (d1[s] << 16);
            }
            for (int t = tid; t < kTN * (kKC / 2); t += kThreads) {
                const int j = t % kTN, kp = (t / kTN) * 2;
                uint32_t d0[kSlices], d1[kSlices];
                const int gk = k0 + kp;
                const bool live = j < nn;
                split_digits(live && gk < K ? lb(gk, n0 + j) : 0.0, c.cexp[j], d0);
                split_digits(live && gk + 1 < K ? lb(gk + 1, n0 + j) : 0.0, c.cexp[j], d1);
                const uint32_t off = core_offset(j, kp);
#pragma unroll
                for (int s = 0; s < kSlices; ++s)
                    *reinterpret_cast<uint32_t*>(c.b_sl + s * kBSliceBytes + off) = d0[s] | (d1[s] << 16);
            }
            fence_proxy_async();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            // ---- 28 digit pairs x 2 K steps of 16, one elected thread
            const bool first_of_drain = (ch % kChunksPerDrain) == 0;
            if (tid == 0 && c.ok) {
                const uint32_t abase = smem_u32(c.a_sl), bbase = smem_u32(c.b_sl);
                for (int ks = 0; ks < kKC / 16; ++ks) {
                    int pair = 0;
                    for (int s = 0; s < kSlices; ++s)
                        for (int t = 0; s + t < kSlices; ++t, ++pair) {
                            const int g = s + t;
                            const uint64_t ad = smem_desc(abase + s * kASliceBytes + ks * 256);
                            const uint64_t bd = smem_desc(bbase + t * kBSliceBytes + ks * 256);
                            // the first product of weight g in this drain group overwrites its accumulator
                            const uint32_t acc = (first_of_drain && ks == 0 && s == 0) ? 0u : 1u;
                            mma_bf16(c.tmem + (uint32_t)(g * kTN), ad, bd, idesc, acc);
                        }
                    (void)pair;
                }
                mma_commit(c.bar);
            }
            if (c.ok && !mbar_wait(c.bar, c.phase)) {
                c.ok = false;
                if (tid == 0) atomicOr(c.status, kErrTimeout);
            }
            c.phase ^= 1u;
            fence_after_sync();
            // ---- read the accumulators back after every kChunksPerDrain chunks and at the end
            if ((ch % kChunksPerDrain) == kChunksPerDrain - 1 || ch == nchunks - 1) {
                const uint32_t lane_base = c.tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
                for (int half = 0; half < kTN / 16; ++half) {
                    long long Hh[16], Hl[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) { Hh[j] = 0; Hl[j] = 0; }
#pragma unroll
                    for (int g = 0; g < kSlices; ++g) {
                        uint32_t v[16];
                        tmem_ld16(lane_base + (uint32_t)(g * kTN + half * 16), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const long long cg = exact_int(v[j]);
                            // Hh = c0 2^21 + c1 2^14 + c2 2^7 + c3; Hl = c4 2^21 + c5 2^14 + c6 2^7 + c7
                            if (g < 4) Hh[j] = Hh[j] * 128 + cg;
                            else Hl[j] = Hl[j] * 128 + cg;
                        }
                    }
                    // H = floor(2^39 sum_g 2^-7g c_g) = Hh 2^18 + floor(Hl 2^-10); the product is
                    // H 2^-39 2^-14 2^(er - 1022) 2^(ec - 1022)
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const long long H = Hh[j] * 262144 + (Hl[j] >> 10);
                        acc[half * 16 + j] += scaled_int(H, er + c.cexp[half * 16 + j] - 2044 - 53);
                    }
                }
                fence_before_sync();
            }
            __syncthreads();
        }
        // ---- epilogue: this thread's row, every column of the tile
        const int r = tid;
        if (r < mm && c.ok) {
#pragma unroll
            for (int j = 0; j < kTN; ++j)
                if (j < nn) epi(m0 + r, n0 + j, acc[j]);
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------------------------------
// Operands split once ("slabs") and multiplied many times: the replay (Algorithm 2) applies the same
// stored factors to every right-hand side of every refinement step, so their digits are computed
// once after the factorisation and kept in device memory in the tensor cores' tile layout. An R x K
// operand becomes, for every K chunk of 32 and every digit s, ceil(R / 8) groups of 8 rows of
// 512 bytes (four 8 x 8 bf16 core matrices): slab byte offset ((kc * kSlices + s) * RG + g) * 512,
// RG = ceil(R / 8). A tile of up to 128 rows of one chunk and digit is thus one contiguous run of
// bytes, copied to shared memory as it is. Rows are scaled by their own power of two (over the
// whole K), kept beside the slab.
// ---------------------------------------------------------------------------------------------------
__host__ __device__ constexpr int64_t slab_bytes(int R, int K) {
    return (int64_t)((K + kKC - 1) / kKC) * kSlices * ((R + 7) / 8) * 512;
}

// Split the R x K operand la(i, k) into a slab (all threads of the block): row exponents first
// (a warp per row), then the digits of element pairs; entries beyond K are zero.
template <class LA>
__device__ void split_to_slab(int R, int K, LA la, uint8_t* slab, int* rexp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int RG = (R + 7) / 8, KC = (K + kKC - 1) / kKC;
    for (int r = warp; r < RG * 8; r += nw) {
        int e = 0;
        if (r < R)
            for (int k = lane; k < K; k += 32) e = max(e, exp_field(la(r, k)));
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (lane == 0) rexp[r] = e;
    }
    __syncthreads();
    const int pairs = RG * 8 * KC * (kKC / 2);
    for (int t = threadIdx.x; t < pairs; t += blockDim.x) {
        const int r = t / (KC * (kKC / 2));
        const int rem = t - r * (KC * (kKC / 2));
        const int kc = rem / (kKC / 2), kp = (rem - kc * (kKC / 2)) * 2;
        const int gk = kc * kKC + kp;
        const int E = rexp[r];
        uint32_t d0[kSlices], d1[kSlices];
        split_digits(r < R && gk < K ? (double)la(r, gk) : 0.0, E, d0);
        split_digits(r < R && gk + 1 < K ? (double)la(r, gk + 1) : 0.0, E, d1);
        const uint32_t within = core_offset(r & 7, kp);   // inside the 512-byte group
#pragma unroll
        for (int sl = 0; sl < kSlices; ++sl)
            *reinterpret_cast<uint32_t*>(slab + (((int64_t)kc * kSlices + sl) * RG + (r >> 3)) * 512 + within) =
                d0[sl] | (d1[sl] << 16);
    }
}

constexpr int kSlabThreads = 256;   // eight warps: two per TMEM lane quarter

// C = A B with A (M x K, rows of a slab whose K chunks start at chunk kc0, RG row groups; row
// exponents rexp) and B from lb(k, j) (K x N, split here per tile). Output tiles of 128 x 32 with
// index tile0 (mod tstride). kSlabThreads threads; the Ctx is set up once per block.
template <class LB, class EPI>
__device__ void tc_gemm_slab(Ctx& c, const uint8_t* aslab, const int* arexp, int RG, int kc0, int M, int N, int K,
                             LB lb, EPI epi, int tile0, int tstride) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tn = (N + kTN - 1) / kTN, tm = (M + kTM - 1) / kTM;
    const uint32_t idesc = instr_desc(kTM, kTN);
    const int quarter = warp & 3, halfc = warp >> 2;   // TMEM lanes 32 quarter.., columns 16 halfc..
    for (int tile = tile0; tile < tm * tn; tile += tstride) {
        const int m0 = (tile / tn) * kTM, n0 = (tile % tn) * kTN;
        const int mm = min(kTM, M - m0), nn = min(kTN, N - n0);
        const int g0 = m0 >> 3, ng = min(kTM / 8, RG - g0);       // row groups of A in this tile
        // column exponents of B over the whole K: eight threads per column
        if (tid < kTN) c.cexp[tid] = 0;
        __syncthreads();
        {
            const int j = tid % kTN, part = tid / kTN, parts = kSlabThreads / kTN;
            int e = 0;
            if (j < nn)
                for (int k = part; k < K; k += parts) e = max(e, exp_field((double)lb(k, n0 + j)));
            if (e) atomicMax(&c.cexp[j], e);
        }
        // the A row groups this tile does not fill must be zero: clear those that may hold data
        if (c.zng > ng) {
            const int nz = c.zng - ng;
            for (int t = tid; t < kSlices * nz * 32; t += kSlabThreads) {
                const int sl = t / (nz * 32), w = t - sl * (nz * 32);
                reinterpret_cast<uint4*>(c.a_sl + sl * kASliceBytes + ng * 512)[w] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        c.zng = ng;
        __syncthreads();
        const int r_mine = quarter * 32 + lane;
        const bool quarter_live = quarter * 32 < mm;          // warp-uniform
        const int er = (r_mine < mm) ? arexp[m0 + r_mine] : 0;
        double acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = 0.0;
        const int nchunks = (K + kKC - 1) / kKC;
        for (int ch = 0; ch < nchunks; ++ch) {
            // A: one contiguous run per digit (16-byte copies)
            const int kc = kc0 + ch;
            for (int t = tid; t < kSlices * ng * 32; t += kSlabThreads) {
                const int sl = t / (ng * 32), w = t - sl * (ng * 32);
                const uint4* src = reinterpret_cast<const uint4*>(aslab + (((int64_t)kc * kSlices + sl) * RG + g0) * 512);
                reinterpret_cast<uint4*>(c.a_sl + sl * kASliceBytes)[w] = __ldg(src + w);
            }
            // B: split the chunk (kTN x kKC) here
            const int k0 = ch * kKC;
            for (int t = tid; t < kTN * (kKC / 2); t += kSlabThreads) {
                const int j = t % kTN, kp = (t / kTN) * 2;
                uint32_t d0[kSlices], d1[kSlices];
                const int gk = k0 + kp;
                const bool live = j < nn;
                split_digits(live && gk < K ? (double)lb(gk, n0 + j) : 0.0, c.cexp[j], d0);
                split_digits(live && gk + 1 < K ? (double)lb(gk + 1, n0 + j) : 0.0, c.cexp[j], d1);
                const uint32_t off = core_offset(j, kp);
#pragma unroll
                for (int sl = 0; sl < kSlices; ++sl)
                    *reinterpret_cast<uint32_t*>(c.b_sl + sl * kBSliceBytes + off) = d0[sl] | (d1[sl] << 16);
            }
            fence_proxy_async();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            const bool first_of_drain = (ch % kChunksPerDrain) == 0;
            if (tid == 0 && c.ok) {
                const uint32_t abase = smem_u32(c.a_sl), bbase = smem_u32(c.b_sl);
                for (int ks = 0; ks < kKC / 16; ++ks)
                    for (int sa = 0; sa < kSlices; ++sa)
                        for (int sb = 0; sa + sb < kSlices; ++sb) {
                            const uint64_t ad = smem_desc(abase + sa * kASliceBytes + ks * 256);
                            const uint64_t bd = smem_desc(bbase + sb * kBSliceBytes + ks * 256);
                            const uint32_t accf = (first_of_drain && ks == 0 && sa == 0) ? 0u : 1u;
                            mma_bf16(c.tmem + (uint32_t)((sa + sb) * kTN), ad, bd, idesc, accf);
                        }
                mma_commit(c.bar);
            }
            if (c.ok && !mbar_wait(c.bar, c.phase)) {
                c.ok = false;
                if (tid == 0) atomicOr(c.status, kErrTimeout);
            }
            c.phase ^= 1u;
            fence_after_sync();
            if (quarter_live && ((ch % kChunksPerDrain) == kChunksPerDrain - 1 || ch == nchunks - 1)) {
                const uint32_t base = c.tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(halfc * 16);
#pragma unroll
                for (int c8 = 0; c8 < 2; ++c8) {
                    long long Hh[8], Hl[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) { Hh[j] = 0; Hl[j] = 0; }
#pragma unroll
                    for (int g = 0; g < kSlices; ++g) {
                        uint32_t v[8];
                        tmem_ld8(base + (uint32_t)(g * kTN + c8 * 8), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const long long cg = exact_int(v[j]);
                            if (g < 4) Hh[j] = Hh[j] * 128 + cg;
                            else Hl[j] = Hl[j] * 128 + cg;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const long long H = Hh[j] * 262144 + (Hl[j] >> 10);
                        acc[c8 * 8 + j] += scaled_int(H, er + c.cexp[halfc * 16 + c8 * 8 + j] - 2044 - 53);
                    }
                }
            }
            fence_before_sync();
            __syncthreads();
        }
        if (r_mine < mm && c.ok) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (halfc * 16 + j < nn) epi(m0 + r_mine, n0 + halfc * 16 + j, acc[j]);
        }
        __syncthreads();
    }
}

}  // namespace tc
}  // namespace ifmm
