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
// scratch entry before reading it, so only the small status word is cleared at each call.  Calls
// whose work overlaps on the GPU (different streams, or the same array reached from several host
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
constexpr int kTileRows = molt::kColTileRows;   // rows per column tile of the sweep kernels
constexpr long long kMaxTileColumns = kStaticScratchFloats / 4;

static __device__ __align__(256) float g_col_scratch[kStaticScratchFloats];
// Bits the column kernels of the last call set when a bounded wait for a tile copy ran out of
// time (their outputs are then incomplete); cleared on the caller's stream at every call.
static __device__ __align__(16) unsigned g_col_status;

constexpr int kMaxDevices = 64;
struct DeviceAddresses {
    float* scratch = nullptr;
    unsigned* status = nullptr;
};
DeviceAddresses g_addr[kMaxDevices];
std::mutex g_addr_mutex;

molt_status noalloc_fail(molt_status s, const std::string& m) {
    molt::set_abi_error(m.c_str());   // reported by molt_last_error(NULL)
    return s;
}

// Device addresses of the two arrays on the current device.  The host-side names g_col_scratch
// and g_col_status are only stand-ins for the symbols and must never be passed to a kernel.
// Outside stream capture the addresses are looked up again on every call, so they follow the
// context that is current (after a cudaDeviceReset, for instance); while `stream` is capturing,
// the addresses of the last call on this device made outside capture are used, so the first call
// on each device must come before any capture.
molt_status device_addresses(cudaStream_t stream, DeviceAddresses* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(MOLT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(MOLT_ERR_UNSUPPORTED, "device index out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        cudaGetLastError();                       // a query error leaves no sticky state
        cap = cudaStreamCaptureStatusActive;      // do not look anything up; use what is known
    }
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        void* q = nullptr;
        e = cudaGetSymbolAddress(&p, g_col_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_col_status);
        if (e != cudaSuccess || p == nullptr || q == nullptr)
            return noalloc_fail(MOLT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev].scratch = static_cast<float*>(p);
        g_addr[dev].status = static_cast<unsigned*>(q);
    } else if (!g_addr[dev].scratch) {
        return noalloc_fail(MOLT_ERR_UNSUPPORTED,
                            "the first allocation-free call on a device must come before any stream capture");
    }
    *out = g_addr[dev];
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
    if (tiles * static_cast<long long>(nx) > kMaxTileColumns)
        return noalloc_fail(MOLT_ERR_ARG, "grid exceeds the static scratch: needs ceil(ny/" + std::to_string(kTileRows) +
                                              ") * nx <= " + std::to_string(kMaxTileColumns) +
                                              " (4 MiB of FP32 scratch)");
    const double h = (bc == molt::BC_PERIODIC) ? Ly / ny : Ly / (ny - 1);
    molt::LineParams<double> lpd;
    const char* err = nullptr;
    if (!molt::build_line_params(c, h, ny, quad_order, bc, &lpd, &err))
        return noalloc_fail(MOLT_ERR_ARG, err ? err : "bad line parameters");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    DeviceAddresses addr;
    molt_status ms = device_addresses(st, &addr);
    if (ms != MOLT_OK) return ms;
    cudaError_t e = cudaMemsetAsync(addr.status, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return noalloc_fail(MOLT_ERR_CUDA, std::string("status reset: ") + cudaGetErrorString(e));
    const long long arr = tiles * nx;
    molt::ColScratch<float> cs;
    cs.aggL = addr.scratch;
    cs.aggR = addr.scratch + arr;
    cs.carL = addr.scratch + 2 * arr;
    cs.carR = addr.scratch + 3 * arr;
    cs.tiles = static_cast<int>(tiles);
    cs.capacity_lines = nx;
    cs.capacity_fields = 1;
    cs.status = addr.status;
    molt::OpArgs<float> a;
    a.in0 = in_dev;
    a.out0 = out_dev;
    const molt::LineParams<float> lp = molt::cast_line_params<float>(lpd);
    e = molt::sweep<float>(1, lp, molt::OP_COPY, a, nx, ny, &cs, nullptr, st, nullptr, nullptr);
    if (e != cudaSuccess) return noalloc_fail(MOLT_ERR_CUDA, std::string("sweep: ") + cudaGetErrorString(e));
    return MOLT_OK;
}

extern "C" molt_status molt_helmholtz_columns_noalloc_status(void* stream, unsigned* status) {
    if (!status) return noalloc_fail(MOLT_ERR_ARG, "null status");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    DeviceAddresses addr;
    molt_status ms = device_addresses(st, &addr);
    if (ms != MOLT_OK) return ms;
    unsigned word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, addr.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(MOLT_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    *status = word;
    return MOLT_OK;
}
