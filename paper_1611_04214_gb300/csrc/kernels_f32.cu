// FP32 instantiation of the sweep, pointwise and reduction kernels.
#include "launch.cuh"

MOLT_INSTANTIATE(float)
