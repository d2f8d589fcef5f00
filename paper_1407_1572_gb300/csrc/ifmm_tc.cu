// ifmm_tc.cu -- the tensor-core FP64 product (ifmm_tc.cuh) as a C-ABI entry point of its own, so that
// its arithmetic can be checked against FP64 products in isolation.
#include <cstdio>

#include "ifmm.h"
#include "ifmm_internal.h"
#include "ifmm_tc.cuh"

namespace ifmm {
namespace {

__device__ int g_tc_status;

__global__ void __launch_bounds__(tc::kThreads, 1)
    k_tc_dgemm(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int M, int N, int K) {
    extern __shared__ __align__(1024) uint8_t tsm[];
    tc::Ctx c;
    tc::ctx_init(c, tsm, &g_tc_status);
    tc::tc_gemm(
        c, M, N, K, [&](int i, int k) { return A[(size_t)i * lda + k]; },
        [&](int k, int j) { return B[(size_t)k * ldb + j]; },
        [&](int i, int j, double v) { C[(size_t)i * ldc + j] = v; }, blockIdx.x, gridDim.x);
    tc::ctx_release(c);
}

}  // namespace
}  // namespace ifmm

extern "C" ifmm_status ifmm_tc_dgemm(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                                     int64_t ldc, int M, int N, int K, void* stream) {
    using namespace ifmm;
    if (!A || !B || !C || M < 0 || N < 0 || K < 0 || lda < K || ldb < N || ldc < N) return IFMM_ERR_INVALID_ARG;
    if ((int64_t)M * ldc >= (1ll << 40)) return IFMM_ERR_INVALID_ARG;
    if (M == 0 || N == 0) return IFMM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    void* sp = nullptr;
    if (cudaGetSymbolAddress(&sp, g_tc_status) != cudaSuccess) return IFMM_ERR_CUDA;
    if (cudaMemsetAsync(sp, 0, sizeof(int), st) != cudaSuccess) return IFMM_ERR_CUDA;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_tc_dgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes) !=
            cudaSuccess)
            return IFMM_ERR_CUDA;
        attr = true;
    }
    const int tiles = ((M + tc::kTM - 1) / tc::kTM) * ((N + tc::kTN - 1) / tc::kTN);
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = tiles < 2 * sms ? tiles : 2 * sms;
    k_tc_dgemm<<<grid, tc::kThreads, tc::kSmemBytes, st>>>(A, (int)lda, B, (int)ldb, C, (int)ldc, M, N, K);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) return IFMM_ERR_CUDA;
    int hs = 0;
    if (cudaMemcpyAsync(&hs, sp, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return IFMM_ERR_CUDA;
    return (hs & tc::kErrTimeout) ? IFMM_ERR_TIMEOUT : IFMM_OK;
}
