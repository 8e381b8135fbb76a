// FP64 instantiation of the vector Cahn-Hilliard sweeps.
#include "vch_sweep.cuh"

MOLT_INSTANTIATE_VCH(double)
