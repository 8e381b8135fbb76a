// FP64 instantiation of the sweep, pointwise and reduction kernels, plus the shared
// fixed-order sum of reduction partials.
#include "launch.cuh"

namespace molt {
namespace detail {

__global__ void sum_partials_kernel(const double* partials, int n, double* result) {
    // one block, fixed order: thread t sums t, t + blockDim, ...; then a fixed tree
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) *result = s;
}

}  // namespace detail

int reduce_blocks() { return detail::kRedBlocks; }

namespace detail {

__global__ void loop_init_kernel(LoopState* ls, unsigned long long* red) {
    ls->k = 0;
    ls->stall = 0;
    ls->done = 0;
    ls->converged = 0;
    ls->best = __longlong_as_double(0x7ff0000000000000LL);   // +inf
    ls->res = ls->best;
    ls->tol_used = 0.0;
    red[0] = 0ull;
    red[1] = 0ull;
}

__global__ void loop_check_kernel(cudaGraphConditionalHandle h, LoopState* ls, unsigned long long* red,
                                  double tol, int max_iter, int fp32) {
    const double res = __longlong_as_double(static_cast<long long>(red[0]));
    const double wmax = __longlong_as_double(static_cast<long long>(red[1]));
    red[0] = 0ull;
    red[1] = 0ull;
    const int k = ls->k + 1;
    ls->k = k;
    const double ulp = wmax * 5.9604644775390625e-08;       // 2^-24 max|w|
    double tol_used = fp32 ? fmax(tol, 2.0 * ulp) : tol;
    bool conv = false, stop = false;
    if (!isfinite(res)) {
        stop = true;
    } else if (res < tol_used) {
        conv = true;
    } else if (res < ls->best) {
        ls->best = res;
        ls->stall = 0;
    } else if (fp32 && res < 64.0 * ulp && ++ls->stall >= 6) {
        conv = true;
        tol_used = res;
    }
    ls->res = res;
    ls->tol_used = tol_used;
    ls->converged = conv ? 1 : 0;
    stop = stop || conv || k >= max_iter;
    ls->done = stop ? 1 : 0;
    cudaGraphSetConditional(h, stop ? 0u : 1u);
}

}  // namespace detail

cudaError_t loop_init(LoopState* ls, unsigned long long* red, cudaStream_t st) {
    detail::loop_init_kernel<<<1, 1, 0, st>>>(ls, red);
    return cudaGetLastError();
}

cudaError_t loop_check(cudaGraphConditionalHandle h, LoopState* ls, unsigned long long* red, double tol, int max_iter,
                       int fp32, cudaStream_t st) {
    detail::loop_check_kernel<<<1, 1, 0, st>>>(h, ls, red, tol, max_iter, fp32);
    return cudaGetLastError();
}

}  // namespace molt

MOLT_INSTANTIATE(double)
