// pipe_peaks.cu -- measured peak rates of the FP64 and FP32 pipes of the current GPU, for the
// roofline denominators of the kernels that run on them (the bench divides each kernel's
// algorithmic flops by its CUDA-event time and by these rates).
//
// Each thread runs long chains of independent fused multiply-adds (eight accumulators, so the
// pipe, not the latency of one chain, bounds the rate) over a grid of several blocks per SM;
// CUDA events on the launching stream time the launch after a warm-up. The result is written to
// device memory so the compiler keeps every operation. Built into its own library
// (libifmm_peaks.so), separate from the solver.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
int time_chain(T* buf, int blocks, int iters, double* tflops) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 2;
    const T a = (T)0.999999, b = (T)1e-7;
    k_fma_chain<T><<<blocks, 256>>>(buf, iters / 4 + 1, a, b);   // warm-up
    cudaEventRecord(e0);
    k_fma_chain<T><<<blocks, 256>>>(buf, iters, a, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || !(ms > 0.f)) return 2;
    const double fmas = (double)blocks * 256.0 * iters * 16.0 * 8.0;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return 0;
}

}  // namespace

extern "C" {

// out[0] = FP64 TFLOP/s, out[1] = FP32 TFLOP/s (fused multiply-add = 2 flops), out[2] = SM count,
// out[3] = SM clock (MHz) reported by the device attributes. Runs on the current device and the
// legacy default stream; returns 0, or 2 on a CUDA failure.
int ifmm_pipe_peaks(double* out) {
    int dev = 0, sms = 0, clk = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 2;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    const int blocks = sms * 8;
    void* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)blocks * 256) != cudaSuccess) return 2;
    double f64 = 0.0, f32 = 0.0;
    int rc = time_chain<double>((double*)buf, blocks, 64, &f64);
    if (rc == 0) rc = time_chain<float>((float*)buf, blocks, 2048, &f32);
    cudaFree(buf);
    if (rc) return rc;
    out[0] = f64;
    out[1] = f32;
    out[2] = sms;
    out[3] = clk / 1000.0;
    return 0;
}

}  // extern "C"
