// peaks.cu -- diagnostics: dense fused-multiply-add throughput of the FP32 and
// FP64 pipes (the denominators of the roofline fractions of the kernels that
// are bound by arithmetic rather than by HBM: the whole-run 1D kernel, the
// complex128 passes), and the failure path of the bounded device-side waits.
#include <cuda_runtime.h>

#include "kernels.h"
#include "tma.cuh"

namespace xsde {
namespace {

// CH independent FMA chains per thread, each converging to the bounded fixed
// point c/(1-b); the data-dependent store keeps them live.
template <typename R, int CH>
__global__ void __launch_bounds__(256) fma_chains_kernel(int iters, R *sink) {
    R a[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = R(1) + R(k) * R(1e-3) + R(threadIdx.x) * R(1e-6);
    const R b = R(0.999), c = R(1e-4);
#pragma unroll 4
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < CH; ++k) a[k] = fma(a[k], b, c);
    R s = R(0);
#pragma unroll
    for (int k = 0; k < CH; ++k) s += a[k];
    if (s == R(-1)) sink[blockIdx.x] = s;
}

template <typename R> int time_chains(int blocks, int iters, double *tflops) {
    constexpr int CH = 8;
    R *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(R) * blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        fma_chains_kernel<R, CH><<<blocks, 256>>>(iters / 4, sink);   // warm-up
        cudaEventRecord(e0);
        fma_chains_kernel<R, CH><<<blocks, 256>>>(iters, sink);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) return -1;
    *tflops = 2.0 * CH * (double)iters * blocks * 256 / (ms * 1e-3) / 1e12;
    return 0;
}

// One CTA waits, with the bounded mbarrier wait of the TMA pipelines, on a
// barrier that expects one arrival nothing makes; when the limit passes it
// records the timeout in the error word, as a pipeline whose copy never lands.
__global__ void wait_timeout_kernel(uint64_t wait_ns, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool landed = mbar_wait(&bar, 0u, wait_ns);
    if (!__syncthreads_and(landed) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_timeout(uint64_t wait_ns, int *status, cudaStream_t s) {
    wait_timeout_kernel<<<1, 32, 0, s>>>(wait_ns, status);
    return cudaGetLastError();
}

int measure_fma_peaks(double *fp32_tflops, double *fp64_tflops) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;   // 64 warps per SM
    if (fp32_tflops && time_chains<float>(blocks, 200000, fp32_tflops) != 0) return -1;
    if (fp64_tflops && time_chains<double>(blocks, 2000, fp64_tflops) != 0) return -1;
    return 0;
}

}  // namespace xsde
