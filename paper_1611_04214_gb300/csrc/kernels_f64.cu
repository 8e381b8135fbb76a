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

}  // namespace molt

MOLT_INSTANTIATE(double)
