// FP32 and FP64 instantiation of the 3D split stage's x-line combination sweep (OpComb3), in a
// translation unit of its own so that it compiles in parallel with the rest.
#include "launch.cuh"

namespace molt {

template <typename T>
cudaError_t sweep_c3(int axis, const LineParams<T>& lp, int kind, const OpArgs<T>& a, int nx, int ny,
                     ColScratch<T>* cs, unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof) {
    return detail::dispatch<T, OpComb3<T>>(axis, lp, a, nx, ny, cs, red, st, launches, prof, kind);
}

template cudaError_t sweep_c3<float>(int, const LineParams<float>&, int, const OpArgs<float>&, int, int,
                                     ColScratch<float>*, unsigned long long*, cudaStream_t, long long*, Prof*);
template cudaError_t sweep_c3<double>(int, const LineParams<double>&, int, const OpArgs<double>&, int, int,
                                      ColScratch<double>*, unsigned long long*, cudaStream_t, long long*, Prof*);

}  // namespace molt
