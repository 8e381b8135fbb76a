// Column (y) Helmholtz sweep that allocates nothing: its scratch lives in a file-scope device
// array instead of solver-owned workspace.
//
// For callers that cannot call cudaMalloc: code running under a memory manager that owns all
// device memory (a framework's caching allocator, a fixed arena), or in a latency-critical loop
// where an allocation or free could synchronize the device.  Such callers still pass their own
// input and output buffers; only the sweep's internal scratch (per-tile segment aggregates and
// carries of the column scan) comes from the static array below.
//
// The array is reserved in every GPU that loads the library and stays there until the process
// exits.  All calls share it and it keeps the last call's contents; each call writes every
// scratch entry before reading it, so nothing has to be cleared between calls.  Calls whose
// work overlaps on the GPU (different streams, or the same array reached from several host
// threads without ordering) race on the array and must be serialized by the caller.
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/molt.h"
#include "molt_internal.h"

namespace {

// 4 MiB of FP32 scratch: aggregates and carries, 4 arrays of tiles x columns floats each.
constexpr long long kStaticScratchFloats = 1LL << 20;
constexpr int kTileRows = 128;   // rows per column tile of the sweep kernels

static __device__ __align__(256) float g_col_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

molt_status noalloc_fail(molt_status s, const std::string& m) {
    molt::set_abi_error(m.c_str());   // reported by molt_last_error(NULL)
    return s;
}

// Device address of the array on the current device, looked up by the first call on each device
// (which should therefore come before any stream capture).  The host-side name g_col_scratch is
// only a stand-in for the symbol and must never be passed to a kernel.
molt_status scratch_address(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(MOLT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(MOLT_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_col_scratch);
        if (e != cudaSuccess || p == nullptr)
            return noalloc_fail(MOLT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return MOLT_OK;
}

}  // namespace

extern "C" molt_status molt_helmholtz_columns_noalloc(int nx, int ny, double Ly, int bc, int quad_order, double c,
                                                      const float* in_dev, float* out_dev, void* stream) {
    if (!in_dev || !out_dev) return noalloc_fail(MOLT_ERR_ARG, "null field");
    if (in_dev == out_dev) return noalloc_fail(MOLT_ERR_ARG, "column sweeps cannot run in place");
    if (nx < 1 || ny < quad_order + 2) return noalloc_fail(MOLT_ERR_ARG, "grid too small for the quadrature order");
    if (!(Ly > 0.0)) return noalloc_fail(MOLT_ERR_ARG, "domain length must be positive");
    const long long tiles = (ny + kTileRows - 1) / kTileRows;
    if (4 * tiles * static_cast<long long>(nx) > kStaticScratchFloats)
        return noalloc_fail(MOLT_ERR_ARG, "grid exceeds the static scratch: needs ceil(ny/128) * nx <= 262144 "
                                          "(4 MiB of FP32 scratch)");
    const double h = (bc == molt::BC_PERIODIC) ? Ly / ny : Ly / (ny - 1);
    molt::LineParams<double> lpd;
    const char* err = nullptr;
    if (!molt::build_line_params(c, h, ny, quad_order, bc, &lpd, &err))
        return noalloc_fail(MOLT_ERR_ARG, err ? err : "bad line parameters");
    float* scratch = nullptr;
    molt_status st = scratch_address(&scratch);
    if (st != MOLT_OK) return st;
    const long long arr = tiles * nx;
    molt::ColScratch<float> cs;
    cs.aggL = scratch;
    cs.aggR = scratch + arr;
    cs.carL = scratch + 2 * arr;
    cs.carR = scratch + 3 * arr;
    cs.tiles = static_cast<int>(tiles);
    cs.capacity_lines = nx;
    cs.capacity_fields = 1;
    molt::OpArgs<float> a;
    a.in0 = in_dev;
    a.out0 = out_dev;
    const molt::LineParams<float> lp = molt::cast_line_params<float>(lpd);
    cudaError_t e = molt::sweep<float>(1, lp, molt::OP_COPY, a, nx, ny, &cs, nullptr,
                                       static_cast<cudaStream_t>(stream), nullptr, nullptr);
    if (e != cudaSuccess) return noalloc_fail(MOLT_ERR_CUDA, std::string("sweep: ") + cudaGetErrorString(e));
    return MOLT_OK;
}
