// Vector Cahn-Hilliard passes (Sec. 5.2): the sweeps whose prologues evaluate the coupled lagged
// term of one component from both state fields.  In FP32 they take the pipelined row kernel and
// the TMA column kernel where those apply (the generic kernels otherwise), and they are profiled
// in the slots of their scalar counterparts.  Vector passes 1 and 2 are instantiated in their own
// translation units (kernels_v1.cu, kernels_v2.cu).
#pragma once
#include "launch.cuh"

namespace molt {

template <typename T>
cudaError_t sweep_vch(int axis, const LineParams<T>& lp, int kind, const OpArgs<T>& a, int nx, int ny,
                      ColScratch<T>* cs, unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof) {
    using namespace detail;
    switch (kind) {
        case OP_V1: return sweep_v1<T>(axis, lp, kind, a, nx, ny, cs, red, st, launches, prof);
        case OP_V2: return sweep_v2<T>(axis, lp, kind, a, nx, ny, cs, red, st, launches, prof);
        case OP_V1A: return dispatch<T, Op1aV<T>>(axis, lp, a, nx, ny, cs, red, st, launches, prof, kind);
    }
    return cudaErrorInvalidValue;
}

}  // namespace molt

#define MOLT_INSTANTIATE_VCH(T)                                                                                   \
    template cudaError_t molt::sweep_vch<T>(int, const molt::LineParams<T>&, int, const molt::OpArgs<T>&, int, int, \
                                            molt::ColScratch<T>*, unsigned long long*, cudaStream_t, long long*,    \
                                            molt::Prof*);
