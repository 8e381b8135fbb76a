// Self-test of the bounded device-side waits (diagnostics; the paper has no counterpart).
//
// The TMA column kernels wait on mbarriers for their tile copies; each wait gives up after a
// fixed time instead of spinning forever, and the kernel then records the timeout in a status
// word that the host reads.  This file launches one block whose wait can never complete (no copy
// is issued and nothing arrives on its barrier) through the same wait routine, so that a test can
// check on a real GPU that the wait returns, the status is set and the context stays usable.
#include <cuda_runtime.h>

#include <string>

#include "../../include/molt.h"
#include "cols_tma.cuh"
#include "molt_internal.h"

namespace {

__global__ void bounded_wait_probe_kernel(unsigned* status, unsigned long long* waited_ns) {
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    molt::mbar_init(&bar, 1);
    molt::mbar_init_fence();
    const unsigned long long t0 = molt::global_ns();
    const bool completed = molt::mbar_wait(&bar, 0u);   // phase 0 never completes
    *waited_ns = molt::global_ns() - t0;
    if (!completed) atomicOr(status, molt::kStatusWaitTimeout);
}

molt_status probe_fail(molt_status s, const std::string& m) {
    molt::set_abi_error(m.c_str());
    return s;
}

}  // namespace

extern "C" molt_status molt_selftest_bounded_wait(int* timed_out, double* waited_seconds) {
    if (!timed_out || !waited_seconds) return probe_fail(MOLT_ERR_ARG, "null output");
    unsigned* status = nullptr;
    unsigned long long* ns = nullptr;
    cudaError_t e = cudaMalloc(&status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&ns, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        bounded_wait_probe_kernel<<<1, 32>>>(status, ns);
        e = cudaGetLastError();
    }
    unsigned st = 0;
    unsigned long long waited = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&waited, ns, sizeof(waited), cudaMemcpyDeviceToHost);
    if (status) cudaFree(status);
    if (ns) cudaFree(ns);
    if (e != cudaSuccess) return probe_fail(MOLT_ERR_CUDA, std::string("bounded-wait probe: ") + cudaGetErrorString(e));
    *timed_out = (st & molt::kStatusWaitTimeout) ? 1 : 0;
    *waited_seconds = static_cast<double>(waited) * 1e-9;
    return MOLT_OK;
}
