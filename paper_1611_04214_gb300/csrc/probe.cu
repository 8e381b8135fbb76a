// Arithmetic-throughput probe (diagnostics; the paper has no counterpart).
//
// Measures the rate of dependent-free fused multiply-adds the GPU sustains in FP32 or FP64, to
// state the FP64 sweeps against the ceiling that binds them: on this part the FP64 FMA rate is a
// small fraction of the FP32 rate, so the FP64 line sweeps are arithmetic-bound, not HBM-bound.
// Every thread runs kChains independent FMA chains for `iters` rounds (no memory traffic inside
// the loop); one FMA counts as two floating-point operations.
#include <cuda_runtime.h>

#include <string>

#include "../../include/molt.h"
#include "molt_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T b, T c, int iters, T* sink) {
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = static_cast<T>(threadIdx.x + i) * static_cast<T>(1e-3);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

molt_status probe_fail(molt_status s, const std::string& m) {
    molt::set_abi_error(m.c_str());
    return s;
}

template <typename T>
cudaError_t run_probe(int blocks, int iters, T* sink, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    // b slightly below 1 and c small keep every chain bounded and away from subnormals
    const T b = static_cast<T>(0.999999), c = static_cast<T>(1e-7);
    fma_probe_kernel<T><<<blocks, kThreads>>>(b, c, iters, sink);   // warm-up
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaEventRecord(e0);
    fma_probe_kernel<T><<<blocks, kThreads>>>(b, c, iters, sink);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return e;
    return cudaEventElapsedTime(ms, e0, e1);
}

}  // namespace

extern "C" molt_status molt_fma_throughput_probe(int precision, double* tflops) {
    if (!tflops || (precision != MOLT_FP32 && precision != MOLT_FP64))
        return probe_fail(MOLT_ERR_ARG, "null output or unknown precision");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return probe_fail(MOLT_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    const int blocks = sms * 8;
    const int iters = precision == MOLT_FP64 ? 4096 : 65536;
    void* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&sink, static_cast<size_t>(blocks) * kThreads * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.0f;
    if (e == cudaSuccess)
        e = precision == MOLT_FP64 ? run_probe<double>(blocks, iters, static_cast<double*>(sink), e0, e1, &ms)
                                   : run_probe<float>(blocks, iters, static_cast<float*>(sink), e0, e1, &ms);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return probe_fail(MOLT_ERR_CUDA, std::string("FMA probe: ") + cudaGetErrorString(e));
    const double flops = 2.0 * kChains * static_cast<double>(iters) * blocks * kThreads;
    *tflops = flops / (static_cast<double>(ms) * 1e-3) / 1e12;
    return MOLT_OK;
}
