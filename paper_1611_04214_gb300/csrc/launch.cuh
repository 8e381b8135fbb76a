// Launch layer: builds the fused op of each pass, picks the launch geometry and dispatches
// on the quadrature order.  Included once per precision (kernels_f32.cu, kernels_f64.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "cols_tma.cuh"
#include "molt_internal.h"
#include "sweep_kernels.cuh"

namespace molt {

namespace detail {

constexpr int kRowMaxSmem = 225 * 1024;   // planning bound (opt-in limit minus static shared memory)
constexpr int kColKY = 16;   // positions per thread in a column tile
constexpr int kColWY = 8;    // warps per column tile
constexpr int kColR = kColKY * kColWY;
static_assert(kColR == kColTileRows, "column tile height must match the scratch sizing constant");

template <typename T>
inline void set_strides(OpBase<T>& o, long long ls, long long ps) {
    o.ls = ls;
    o.ps = ps;
}

template <typename T> inline OpCopy<T> build(const OpArgs<T>& a, OpCopy<T>*) {
    OpCopy<T> o; o.in = a.in0; o.out = a.out0; return o;
}
template <typename T> inline OpP1<T> build(const OpArgs<T>& a, OpP1<T>*) {
    OpP1<T> o; o.w = a.in0; o.t_out = a.out0; o.s_out = a.out1; o.g2 = a.g2; o.g1 = a.g1; return o;
}
template <typename T> inline OpP2<T> build(const OpArgs<T>& a, OpP2<T>*) {
    OpP2<T> o; o.w = a.in0; o.t_in = a.in1; o.s_in = a.in2; o.p_out = a.out0; o.u_out = a.out1;
    o.g2 = a.g2; o.g1 = a.g1; o.beta = a.beta; return o;
}
template <typename T> inline OpP3<T> build(const OpArgs<T>& a, OpP3<T>*) {
    OpP3<T> o; o.p_in = a.in0; o.u_in = a.in1; o.q1_out = a.out0; o.q2_out = a.out1; return o;
}
template <typename T> inline OpP4<T> build(const OpArgs<T>& a, OpP4<T>*) {
    OpP4<T> o; o.q1_in = a.in0; o.q2_in = a.in1; o.u_in = a.in2; o.y_in = a.in3; o.w = a.out0;
    o.shift = a.shift; return o;
}
template <typename T> inline Op1a<T> build(const OpArgs<T>& a, Op1a<T>*) {
    Op1a<T> o; o.w = a.in0; o.e_out = a.out0; o.g2 = a.g2; o.g1 = a.g1; o.beta = a.beta; return o;
}
template <typename T> inline Op1b<T> build(const OpArgs<T>& a, Op1b<T>*) {
    Op1b<T> o; o.e_in = a.in0; o.y_in = a.in1; o.w = a.out0; o.shift = a.shift; return o;
}
template <typename T> inline OpP1V<T> build(const OpArgs<T>& a, OpP1V<T>*) {
    OpP1V<T> o; o.v1 = a.in0; o.v2 = a.in1; o.t_out = a.out0; o.s_out = a.out1; o.s = a.vs; o.comp = a.comp;
    return o;
}
template <typename T> inline OpP2V<T> build(const OpArgs<T>& a, OpP2V<T>*) {
    OpP2V<T> o; o.v1 = a.in0; o.v2 = a.in1; o.t_in = a.in2; o.s_in = a.in3; o.p_out = a.out0; o.u_out = a.out1;
    o.s = a.vs; o.beta = a.beta; o.comp = a.comp; return o;
}
template <typename T> inline OpComb3<T> build(const OpArgs<T>& a, OpComb3<T>*) {
    OpComb3<T> o; o.y = a.in0; o.z = a.in1; o.yz = a.in2; o.out = a.out0; o.ka = a.g2; o.kb = a.g1; o.kc = a.beta;
    return o;
}
template <typename T> inline Op1aV<T> build(const OpArgs<T>& a, Op1aV<T>*) {
    Op1aV<T> o; o.v1 = a.in0; o.v2 = a.in1; o.e_out = a.out0; o.s = a.vs; o.beta = a.beta; o.comp = a.comp;
    return o;
}

// Opt the kernel into the largest dynamic shared memory the device allows next to its static
// shared memory; returns that limit (bytes) or -1 on error.
template <class Kern>
int smem_optin(Kern kern) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return -1;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return -1;
    const int limit = optin - static_cast<int>(fa.sharedSizeBytes);
    if (limit <= 0) return -1;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess) return -1;
    return limit;
}

inline int next_pow2_log2(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

inline void prof_begin(Prof* p, int slot, cudaStream_t st) {
    if (p && p->on) p->begin(slot, st);
}
inline void prof_end(Prof* p, cudaStream_t st) {
    if (p && p->on) p->end(st);
}

template <typename T, int M, class Op>
cudaError_t rows(const LineParams<T>& lp, const Op& op, int nlines, unsigned long long* red, cudaStream_t st,
                 Prof* prof, int kind) {
    constexpr int NF = Op::NF;
    const int n = lp.n;
    const int pitch = n + (n >> 5) + 1;
    if (n <= 8192) {
        constexpr int K = 8;
        const int tl_log2 = next_pow2_log2((n + K - 1) / K);
        const int TL = 1 << tl_log2;
        const int threads = TL < 128 ? 128 : TL;
        int lpb = threads / TL;
        while (lpb > 1 && static_cast<long long>(lpb) * NF * pitch * sizeof(T) > 48 * 1024) lpb >>= 1;
        const int block = lpb * TL < 32 ? 32 : lpb * TL;
        const size_t smem = static_cast<size_t>(lpb) * NF * pitch * sizeof(T);
        auto kern = rows_kernel<T, M, K, Op>;
        static int limit = smem_optin(kern);
        if (limit < 0 || smem > static_cast<size_t>(limit)) return cudaErrorInvalidValue;
        const int grid = (nlines + lpb - 1) / lpb;
        prof_begin(prof, kind, st);
        kern<<<grid, block, smem, st>>>(lp, op, nlines, tl_log2, lpb, pitch, red);
        prof_end(prof, st);
    } else if constexpr (NF == 1) {
        constexpr int K = 16;
        const int tl_log2 = next_pow2_log2((n + K - 1) / K);
        const int TL = 1 << tl_log2;
        if (TL > 1024) return cudaErrorInvalidValue;
        const size_t smem = static_cast<size_t>(NF) * pitch * sizeof(T);
        auto kern = rows_kernel<T, M, K, Op>;
        static int limit = smem_optin(kern);
        if (limit < 0 || smem > static_cast<size_t>(limit)) return cudaErrorInvalidValue;
        prof_begin(prof, kind, st);
        kern<<<nlines, TL, smem, st>>>(lp, op, nlines, tl_log2, 1, pitch, red);
        prof_end(prof, st);
    } else {
        return cudaErrorInvalidValue;   // two-field rows are limited to 8192 nodes
    }
    return cudaGetLastError();
}

template <typename T, int M, class Op>
cudaError_t cols(const LineParams<T>& lp, const Op& op, int nlines, ColScratch<T>* cs,
                 unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof, int kind) {
    constexpr int NF = Op::NF;
    const int n = lp.n;
    const int tiles = (n + kColR - 1) / kColR;
    if (cs == nullptr || cs->capacity_lines < nlines || cs->capacity_fields < NF || cs->tiles < tiles)
        return cudaErrorInvalidValue;
    dim3 block(32, kColWY);
    dim3 grid((nlines + 31) / 32, tiles);
    prof_begin(prof, 8 + kind, st);
    cols_agg_kernel<T, M, kColKY, kColWY, Op><<<grid, block, 0, st>>>(lp, op, nlines, cs->aggL, cs->aggR, tiles);
    prof_end(prof, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int total = nlines * NF;
    prof_begin(prof, 16, st);
    cols_carry_kernel<T><<<(total + 127) / 128, 128, 0, st>>>(lp, nlines, NF, tiles, kColR, cs->aggL, cs->aggR,
                                                             cs->carL, cs->carR);
    prof_end(prof, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin(prof, 17 + kind, st);
    cols_final_kernel<T, M, kColKY, kColWY, Op><<<grid, block, 0, st>>>(lp, op, nlines, cs->carL, cs->carR, tiles, red);
    prof_end(prof, st);
    if (launches) *launches += 2;   // the caller counts one
    return cudaGetLastError();
}

// Interior weights duplicated into both halves of a 64-bit word (packed FP32x2 stencil steps).
inline PackedStencil packed_stencil(const LineParams<float>& lp) {
    PackedStencil p;
    std::memset(&p, 0, sizeof(p));
    for (int o = 0; o < kMaxStencil; ++o) {
        unsigned bl, br;
        std::memcpy(&bl, &lp.wl[o], 4);
        std::memcpy(&br, &lp.wr[o], 4);
        p.wl[o] = (static_cast<unsigned long long>(bl) << 32) | bl;
        p.wr[o] = (static_cast<unsigned long long>(br) << 32) | br;
    }
    return p;
}

// ---- pipelined FP32 rows: pointwise op for each row pass ----
template <class Op> struct PipeOf { using type = void; };
template <> struct PipeOf<OpCopy<float>> { using type = PipeCopy<float>; };
template <> struct PipeOf<OpP2<float>> { using type = PipeP2<float>; };
template <> struct PipeOf<OpP4<float>> { using type = PipeP4<float>; };
template <> struct PipeOf<Op1a<float>> { using type = Pipe1a<float>; };
template <> struct PipeOf<OpComb3<float>> { using type = PipeComb3<float>; };
template <> struct PipeOf<Op1b<float>> { using type = Pipe1b<float>; };
template <> struct PipeOf<OpP2V<float>> { using type = PipeP2V<float>; };
template <> struct PipeOf<Op1aV<float>> { using type = Pipe1aV<float>; };

// vector CH pipe forms carry (c1 + c2)/tau and the component; the scalar ones do not
template <class P> inline void set_vch(P&, const OpArgs<float>&) {}
inline void set_vch(PipeP2V<float>& p, const OpArgs<float>& a) { p.vs = a.vs; p.comp = a.comp; }
inline void set_vch(Pipe1aV<float>& p, const OpArgs<float>& a) { p.vs = a.vs; p.comp = a.comp; }
inline void set_vch(PipeP1V<float>& p, const OpArgs<float>& a) { p.vs = a.vs; p.comp = a.comp; }

template <class P>
P pipe_build(int kind, const OpArgs<float>& a) {
    P p{};
    p.g2 = a.g2;
    p.g1 = a.g1;
    p.beta = a.beta;
    switch (kind) {
        case OP_COPY: p.s[0] = a.in0; p.o[0] = a.out0; break;
        case OP_P2: p.s[0] = a.in0; p.s[1] = a.in1; p.s[2] = a.in2; p.o[0] = a.out0; p.o[1] = a.out1; break;
        case OP_P4: p.s[0] = a.in0; p.s[1] = a.in2; p.a[0] = a.out0; p.a[1] = a.in3; p.a[2] = a.in1; p.o[0] = a.out0; break;
        case OP_1A: p.s[0] = a.in0; p.o[0] = a.out0; break;
        case OP_1B: p.s[0] = a.in0; p.a[0] = a.out0; p.a[1] = a.in1; p.o[0] = a.out0; break;
        case OP_V2:
            p.s[0] = a.in0; p.s[1] = a.in1; p.s[2] = a.in2; p.s[3] = a.in3; p.o[0] = a.out0; p.o[1] = a.out1;
            break;
        case OP_V1A: p.s[0] = a.in0; p.s[1] = a.in1; p.o[0] = a.out0; break;
        case OP_C3: p.s[0] = a.in0; p.s[1] = a.in1; p.s[2] = a.in2; p.o[0] = a.out0; break;
    }
    set_vch(p, a);
    return p;
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Shared memory of one block of the pipelined row kernels: the double-buffered staged fields and
// the auxiliary fields of its line (C = 1), or of its slice with a halo chunk on each side padded
// to 8 chunks (the cluster kernel, C = 2).
template <class P>
long long pipe_smem(int n, int C) {
    const long long nchl = n / 4 / C;
    if (C == 1) return (2LL * P::NS + P::NA) * n * 4;
    return (2LL * P::NS * (nchl + 8) + static_cast<long long>(P::NA) * nchl) * 16;
}

// Cluster sizes the pipelined row kernel can run a line of n nodes with: slices of whole warps of
// 16-position threads (n % (512 C) == 0), at most 512 threads per block, and shared memory that fits.
template <class P>
bool pipe_fits(int n, int C) {
    if (n < 1024 || n % (512 * C) != 0 || n / (16 * C) > 512) return false;
    return pipe_smem<P>(n, C) <= kRowMaxSmem;
}

// The cluster size of a line length: MOLT_ROWS_CLUSTER (1 or 2) in the environment when it
// fits, else the smallest that fits; 0 when none does (or a field is not 16-byte aligned).
template <class P>
int pipe_cluster(const P& p, int n) {
    for (int f = 0; f < P::NS; ++f) if (!aligned16(p.s[f])) return 0;
    for (int f = 0; f < P::NA; ++f) if (!aligned16(p.a[f])) return 0;
    for (int f = 0; f < P::NO; ++f) if (!aligned16(p.o[f])) return 0;
    if (const char* v = std::getenv("MOLT_ROWS_CLUSTER")) {
        const int c = std::atoi(v);
        if ((c == 1 || c == 2) && pipe_fits<P>(n, c)) return c;
    }
    for (int c : {1, 2})
        if (pipe_fits<P>(n, c)) return c;
    return 0;
}

// One-block-per-line pipelined row kernel with K positions per thread (n / K threads).
template <int M, class P, int K>
cudaError_t rows_pipe_one(const LineParams<float>& lp, const PackedStencil& pw, const P& op, int nlines, long long ld,
                          size_t smem, unsigned long long* red, cudaStream_t st, Prof* prof, int kind, int rev) {
    const int TL = lp.n / K;
    auto kern = rows_pipe_kernel<M, P, K>;
    static int limit = smem_optin(kern);
    if (limit < 0 || smem > static_cast<size_t>(limit)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TL, smem);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sms * per_sm;
    if (grid > nlines) grid = nlines;
    prof_begin(prof, kind, st);
    kern<<<grid, TL, smem, st>>>(lp, pw, op, nlines, ld, red, rev);
    prof_end(prof, st);
    return cudaGetLastError();
}

template <int M, class P, int C>
cudaError_t rows_pipe(const LineParams<float>& lp, const P& op, int nlines, unsigned long long* red, cudaStream_t st,
                      Prof* prof, int kind, int order) {
    const int n = lp.n;
    const int TL = n / (16 * C);
    const size_t smem = static_cast<size_t>(pipe_smem<P>(n, C));
    const PackedStencil pw = packed_stencil(lp);
    const long long ld = n;
    if constexpr (C == 1) {
        // single-field copy sweeps of lines of at least 4096 nodes: 32 positions per thread (half
        // the warps, about 115 registers), so two blocks share an SM and two lines are in flight
        // (8192 nodes: 146 -> 124 us per 8192^2 sweep); MOLT_ROWS_K32=0 keeps 16
        if constexpr (std::is_same<P, PipeCopy<float>>::value) {
            const char* v = std::getenv("MOLT_ROWS_K32");
            if (!(v && v[0] == '0') && n >= 4096 && n % 1024 == 0)
                return rows_pipe_one<M, P, 32>(lp, pw, op, nlines, ld, smem, red, st, prof, kind, order & 1);
        }
        // otherwise 16 positions per thread (8 for lines of at most 4096 nodes, with twice the
        // warps per block, measured slower)
        return rows_pipe_one<M, P, 16>(lp, pw, op, nlines, ld, smem, red, st, prof, kind, order & 1);
    } else {
        auto kern = rows_cluster_kernel<M, P, C>;
        static int limit = smem_optin(kern);
        if (limit < 0 || smem > static_cast<size_t>(limit)) return cudaErrorInvalidValue;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(TL);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(C * 1024);
        int clusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (clusters < 1) return cudaErrorInvalidConfiguration;
        if (clusters > nlines) clusters = nlines;
        cfg.gridDim = dim3(C * clusters);
        prof_begin(prof, kind, st);
        e = cudaLaunchKernelEx(&cfg, kern, lp, pw, op, nlines, ld, red);
        prof_end(prof, st);
        return e;
    }
}

// ---- pipelined FP32 columns ----
template <class Op> struct ColPipeOf { using type = void; };
template <> struct ColPipeOf<OpCopy<float>> { using type = PipeCopy<float>; };
template <> struct ColPipeOf<OpP1<float>> { using type = PipeP1<float>; };
template <> struct ColPipeOf<OpP3<float>> { using type = PipeP3<float>; };
template <> struct ColPipeOf<OpP1V<float>> { using type = PipeP1V<float>; };

template <class P>
P col_pipe_build(int kind, const OpArgs<float>& a) {
    P p{};
    p.g2 = a.g2;
    p.g1 = a.g1;
    p.beta = a.beta;
    switch (kind) {
        case OP_COPY: p.s[0] = a.in0; p.o[0] = a.out0; break;
        case OP_P1: p.s[0] = a.in0; p.o[0] = a.out0; p.o[1] = a.out1; break;
        case OP_P3: p.s[0] = a.in0; p.s[1] = a.in1; p.o[0] = a.out0; p.o[1] = a.out1; break;
        case OP_V1: p.s[0] = a.in0; p.s[1] = a.in1; p.o[0] = a.out0; p.o[1] = a.out1; break;
    }
    set_vch(p, a);
    return p;
}

template <class P>
bool col_pipe_eligible(const P& p, int n, int nlines) {
    if (nlines % 32 != 0 || n < 256) return false;
    for (int f = 0; f < P::NS; ++f) if (!aligned16(p.s[f])) return false;
    return true;
}

template <int M, class P, bool kFinal>
cudaError_t cols_pipe_launch(const LineParams<float>& lp, const P& op, int nlines, int tiles, ColScratch<float>* cs,
                             unsigned long long* red, cudaStream_t st) {
    constexpr int ROWS = kColR + 2 * (kMaxM / 2);
    const size_t smem = static_cast<size_t>(2) * P::NS * ROWS * 32 * sizeof(float);
    auto kern = cols_pipe_kernel<M, P, kFinal>;
    static int limit = smem_optin(kern);
    if (limit < 0 || smem > static_cast<size_t>(limit)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kColWY, smem);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int items = (nlines / 32) * tiles;
    int grid = sms * per_sm;
    if (grid > items) grid = items;
    kern<<<grid, 32 * kColWY, smem, st>>>(lp, op, nlines, static_cast<long long>(nlines), tiles, cs->aggL, cs->aggR,
                                          cs->carL, cs->carR, red);
    return cudaGetLastError();
}

template <int M, class P>
cudaError_t cols_pipe(const LineParams<float>& lp, const P& op, int nlines, ColScratch<float>* cs,
                      unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof, int kind) {
    const int n = lp.n;
    const int tiles = (n + kColR - 1) / kColR;
    if (cs == nullptr || cs->capacity_lines < nlines || cs->capacity_fields < P::NF || cs->tiles < tiles)
        return cudaErrorInvalidValue;
    prof_begin(prof, 8 + kind, st);
    cudaError_t e = cols_pipe_launch<M, P, false>(lp, op, nlines, tiles, cs, red, st);
    prof_end(prof, st);
    if (e != cudaSuccess) return e;
    const int strips = (nlines + 31) / 32;
    prof_begin(prof, 16, st);
    cols_carry_split_kernel<float><<<P::NF * strips, dim3(32, 8), 0, st>>>(lp, nlines, P::NF, tiles, kColR, cs->aggL,
                                                                          cs->aggR, cs->carL, cs->carR);
    prof_end(prof, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin(prof, 17 + kind, st);
    e = cols_pipe_launch<M, P, true>(lp, op, nlines, tiles, cs, red, st);
    prof_end(prof, st);
    if (launches) *launches += 2;
    return e;
}

// ---- FP32 columns with TMA tile loads (cols_tma.cuh) ----
// The driver's tensor-map encoder, looked up once through the runtime (no link against libcuda).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// TMA column kernels are the default for eligible FP32 column sweeps; MOLT_COLS_TMA=0 in the
// environment at launch (or graph capture) time selects the cp.async kernels instead.  Both
// evaluate the same operations in the same order, so their results agree bit for bit.
inline bool cols_tma_enabled() {
    const char* v = std::getenv("MOLT_COLS_TMA");
    return !(v && v[0] == '0');
}

// One map per staged field: an n x nlines row-major FP32 array, box of 32 columns x rows rows.
template <class P>
bool col_tma_maps(const P& op, int nlines, int n, int rows, ColMaps* maps) {
    std::memset(maps, 0, sizeof(*maps));
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    for (int f = 0; f < P::NS; ++f) {
        const cuuint64_t dims[2] = {static_cast<cuuint64_t>(nlines), static_cast<cuuint64_t>(n)};
        const cuuint64_t strides[1] = {static_cast<cuuint64_t>(nlines) * sizeof(float)};
        const cuuint32_t box[2] = {32u, static_cast<cuuint32_t>(rows)};
        const cuuint32_t estr[2] = {1u, 1u};
        if (enc(&maps->m[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(op.s[f]), dims, strides, box,
                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}


template <int M, class P, bool kFinal>
cudaError_t cols_tma_launch(const LineParams<float>& lp, const ColMaps& maps, const PackedStencil& pw, const P& op,
                            int nlines, int tiles, ColScratch<float>* cs, unsigned long long* red, cudaStream_t st,
                            int rev) {
    constexpr int ROWS = kColR + M;
    const size_t smem = static_cast<size_t>(tma_col_stages(P::NS)) * P::NS * ROWS * 32 * sizeof(float) + 128;
    auto kern = cols_tma_kernel<M, P, kFinal>;
    static int limit = smem_optin(kern);
    if (limit < 0 || smem > static_cast<size_t>(limit)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kColWY, smem);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int items = (nlines / 32) * tiles;
    int grid = sms * per_sm;
    if (grid > items) grid = items;
    kern<<<grid, 32 * kColWY, smem, st>>>(lp, maps, pw, op, nlines, static_cast<long long>(nlines), tiles, cs->aggL,
                                          cs->aggR, cs->carL, cs->carR, cs->status, red, rev);
    count_tma_launch();
    return cudaGetLastError();
}

template <int M, class P>
cudaError_t cols_tma(const LineParams<float>& lp, const ColMaps& maps, const P& op, int nlines, ColScratch<float>* cs,
                     unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof, int kind, int order) {
    const int n = lp.n;
    const int tiles = (n + kColR - 1) / kColR;
    if (cs == nullptr || cs->capacity_lines < nlines || cs->capacity_fields < P::NF || cs->tiles < tiles)
        return cudaErrorInvalidValue;
    const PackedStencil pw = packed_stencil(lp);
    prof_begin(prof, 8 + kind, st);
    cudaError_t e = cols_tma_launch<M, P, false>(lp, maps, pw, op, nlines, tiles, cs, red, st, order & 1);
    prof_end(prof, st);
    if (e != cudaSuccess) return e;
    const int strips = (nlines + 31) / 32;
    prof_begin(prof, 16, st);
    cols_carry_split_kernel<float><<<P::NF * strips, dim3(32, 8), 0, st>>>(lp, nlines, P::NF, tiles, kColR, cs->aggL,
                                                                          cs->aggR, cs->carL, cs->carR);
    prof_end(prof, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prof_begin(prof, 17 + kind, st);
    e = cols_tma_launch<M, P, true>(lp, maps, pw, op, nlines, tiles, cs, red, st, (order >> 1) & 1);
    prof_end(prof, st);
    if (launches) *launches += 2;
    return e;
}

// The alternating block orders of the 2D iteration (OpArgs::order) are on by default;
// MOLT_BLOCK_ORDER=0 in the environment at launch (or graph capture) time runs every pass from the
// first line / tile row down.  Results do not depend on it.
inline bool block_order_enabled() {
    const char* v = std::getenv("MOLT_BLOCK_ORDER");
    return !(v && v[0] == '0');
}

template <typename T, class Op>
cudaError_t dispatch(int axis, const LineParams<T>& lp, const OpArgs<T>& a_in, int nx, int ny, ColScratch<T>* cs,
                     unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof, int kind) {
    OpArgs<T> a = a_in;
    if (!block_order_enabled()) a.order = 0;
    Op op = build(a, static_cast<Op*>(nullptr));
    // the vector CH passes are timed in the slots of their scalar counterparts
    const int pk = kind == OP_V1 ? OP_P1 : kind == OP_V2 ? OP_P2 : kind == OP_V1A ? OP_1A : kind == OP_C3 ? OP_COPY
                                                                                                        : kind;
    const int nlines = axis == 0 ? ny : nx;
    set_strides<T>(op, axis == 0 ? nx : 1, axis == 0 ? 1 : nx);
    if (launches) *launches += 1;
    if (axis == 0) {
        if (a.variant >= LAUNCH_COLS_TMA) return cudaErrorInvalidValue;
        if constexpr (std::is_same<T, float>::value && !std::is_same<typename PipeOf<Op>::type, void>::value) {
            using P = typename PipeOf<Op>::type;
            const P pop = pipe_build<P>(kind, a);
            int C = a.variant == LAUNCH_ROWS_GENERAL ? 0 : pipe_cluster(pop, lp.n);
            if (a.variant == LAUNCH_ROWS_ONE_BLOCK || a.variant == LAUNCH_ROWS_CLUSTER2) {
                C = a.variant == LAUNCH_ROWS_ONE_BLOCK ? 1 : 2;
                if (pipe_cluster(pop, lp.n) == 0 || !pipe_fits<P>(lp.n, C)) return cudaErrorInvalidValue;
            }
            if (C > 0) {
                switch (lp.M * 8 + C) {
                    case 2 * 8 + 1: return rows_pipe<2, P, 1>(lp, pop, nlines, red, st, prof, pk, a.order);
                    case 2 * 8 + 2: return rows_pipe<2, P, 2>(lp, pop, nlines, red, st, prof, pk, a.order);
                    case 4 * 8 + 1: return rows_pipe<4, P, 1>(lp, pop, nlines, red, st, prof, pk, a.order);
                    case 4 * 8 + 2: return rows_pipe<4, P, 2>(lp, pop, nlines, red, st, prof, pk, a.order);
                    case 6 * 8 + 1: return rows_pipe<6, P, 1>(lp, pop, nlines, red, st, prof, pk, a.order);
                    case 6 * 8 + 2: return rows_pipe<6, P, 2>(lp, pop, nlines, red, st, prof, pk, a.order);
                }
            }
        }
        if (a.variant == LAUNCH_ROWS_ONE_BLOCK || a.variant == LAUNCH_ROWS_CLUSTER2) return cudaErrorInvalidValue;
        if constexpr ((Op::kAxes & 1) != 0) {
            switch (lp.M) {
                case 2: return rows<T, 2>(lp, op, nlines, red, st, prof, pk);
                case 4: return rows<T, 4>(lp, op, nlines, red, st, prof, pk);
                case 6: return rows<T, 6>(lp, op, nlines, red, st, prof, pk);
            }
        }
    } else {
        if (a.variant != LAUNCH_DEFAULT && a.variant < LAUNCH_COLS_TMA) return cudaErrorInvalidValue;
        if (a.variant == LAUNCH_ROWS_TENSOR_CORE) return cudaErrorInvalidValue;
        if constexpr (std::is_same<T, float>::value && !std::is_same<typename ColPipeOf<Op>::type, void>::value) {
            using P = typename ColPipeOf<Op>::type;
            const P pop = col_pipe_build<P>(kind, a);
            const bool eligible = col_pipe_eligible(pop, lp.n, nlines);
            if (!eligible && (a.variant == LAUNCH_COLS_TMA || a.variant == LAUNCH_COLS_CP_ASYNC))
                return cudaErrorInvalidValue;
            if (eligible && a.variant != LAUNCH_COLS_GENERAL) {
                ColMaps maps;
                const bool want_tma = a.variant == LAUNCH_COLS_TMA || (a.variant == LAUNCH_DEFAULT && cols_tma_enabled());
                const bool have_maps = want_tma && col_tma_maps(pop, nlines, lp.n, kColR + lp.M, &maps);
                if (a.variant == LAUNCH_COLS_TMA && !have_maps) return cudaErrorInvalidValue;
                if (have_maps) {
                    switch (lp.M) {
                        case 2: return cols_tma<2>(lp, maps, pop, nlines, cs, red, st, launches, prof, pk, a.order);
                        case 4: return cols_tma<4>(lp, maps, pop, nlines, cs, red, st, launches, prof, pk, a.order);
                        case 6: return cols_tma<6>(lp, maps, pop, nlines, cs, red, st, launches, prof, pk, a.order);
                    }
                }
                switch (lp.M) {
                    case 2: return cols_pipe<2>(lp, pop, nlines, cs, red, st, launches, prof, pk);
                    case 4: return cols_pipe<4>(lp, pop, nlines, cs, red, st, launches, prof, pk);
                    case 6: return cols_pipe<6>(lp, pop, nlines, cs, red, st, launches, prof, pk);
                }
            }
        }
        if (a.variant == LAUNCH_COLS_TMA || a.variant == LAUNCH_COLS_CP_ASYNC) return cudaErrorInvalidValue;
        if constexpr ((Op::kAxes & 2) != 0) {
            switch (lp.M) {
                case 2: return cols<T, 2>(lp, op, nlines, cs, red, st, launches, prof, pk);
                case 4: return cols<T, 4>(lp, op, nlines, cs, red, st, launches, prof, pk);
                case 6: return cols<T, 6>(lp, op, nlines, cs, red, st, launches, prof, pk);
            }
        }
    }
    return cudaErrorInvalidValue;
}

// ---- pointwise and reductions ----
// out = c0 x0 + c1 x1 + c2 x2 + c3 x3 + c4 in the field precision (FP64 arithmetic on an FP32
// field would make this pass ALU-bound on a part with a small FP64 rate).
template <typename T>
__device__ __forceinline__ T lin_elem(const T* x0, T c0, const T* x1, T c1, const T* x2, T c2, const T* x3, T c3,
                                      T c4, long long i) {
    if (x0 && x1 && c1 == -c0 && !x2 && !x3) return fma(c0, x0[i] - x1[i], c4);   // scaled difference
    T acc = c4;
    if (x0) acc = fma(c0, x0[i], acc);
    if (x1) acc = fma(c1, x1[i], acc);
    if (x2) acc = fma(c2, x2[i], acc);
    if (x3) acc = fma(c3, x3[i], acc);
    return acc;
}

template <typename T>
__global__ void lincomb_kernel(T* out, long long n, const T* x0, T c0, const T* x1, T c1, const T* x2, T c2,
                               const T* x3, T c3, T c4) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n; i += stride)
        out[i] = lin_elem(x0, c0, x1, c1, x2, c2, x3, c3, c4, i);
}

// FP32 with every pointer 16-byte aligned and n % 4 == 0: four elements per thread and access.
static __global__ void lincomb4_kernel(float* out, long long n4, const float* x0, float c0, const float* x1, float c1,
                                const float* x2, float c2, const float* x3, float c3, float c4) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n4; i += stride) {
        float4 acc = make_float4(c4, c4, c4, c4);
        if (x1 && c1 == -c0 && !x2 && !x3) {
            // scaled difference c0 (x0 - x1): difference first (exact for nearby values), then scale
            const float4 a = reinterpret_cast<const float4*>(x0)[i];
            const float4 b = reinterpret_cast<const float4*>(x1)[i];
            acc.x = fmaf(c0, a.x - b.x, c4);
            acc.y = fmaf(c0, a.y - b.y, c4);
            acc.z = fmaf(c0, a.z - b.z, c4);
            acc.w = fmaf(c0, a.w - b.w, c4);
            reinterpret_cast<float4*>(out)[i] = acc;
            continue;
        }
        auto add = [&](const float* x, float c) {
            if (!x) return;
            const float4 v = reinterpret_cast<const float4*>(x)[i];
            acc.x = fmaf(c, v.x, acc.x);
            acc.y = fmaf(c, v.y, acc.y);
            acc.z = fmaf(c, v.z, acc.z);
            acc.w = fmaf(c, v.w, acc.w);
        };
        add(x0, c0);
        add(x1, c1);
        add(x2, c2);
        add(x3, c3);
        reinterpret_cast<float4*>(out)[i] = acc;
    }
}

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double s[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kRedThreads / 32; ++i) r += s[i];
    return r;
}

// which = 0: energy, 1: mass (trapezoid weights 1/2 on non-periodic wall nodes).
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
energy_mass_kernel(const T* u, int nx, int ny, int bc, double hx, double hy, double eps, int which, double* partials) {
    const long long total = static_cast<long long>(nx) * ny;
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    const bool periodic = bc == BC_PERIODIC;
    const double e2 = 0.5 * eps * eps;
    double acc = 0.0;
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total; idx += stride) {
        const int i = static_cast<int>(idx % nx);
        const int j = static_cast<int>(idx / nx);
        const double wx = (!periodic && (i == 0 || i == nx - 1)) ? 0.5 : 1.0;
        const double wy = (ny == 1) ? 1.0 : ((!periodic && (j == 0 || j == ny - 1)) ? 0.5 : 1.0);
        const double x = static_cast<double>(u[idx]);
        if (which == 1) {
            acc += wx * wy * x;
            continue;
        }
        const double q = x * x - 1.0;
        acc += wx * wy * 0.25 * q * q;
        if (periodic || i < nx - 1) {
            const int i1 = (i + 1 == nx) ? 0 : i + 1;
            const double g = (static_cast<double>(u[static_cast<long long>(j) * nx + i1]) - x) / hx;
            acc += wy * e2 * g * g;
        }
        if (ny > 1 && (periodic || j < ny - 1)) {
            const int j1 = (j + 1 == ny) ? 0 : j + 1;
            const double g = (static_cast<double>(u[static_cast<long long>(j1) * nx + i]) - x) / hy;
            acc += wx * e2 * g * g;
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s * hx * (ny == 1 ? 1.0 : hy);
}

__global__ void sum_partials_kernel(const double* partials, int n, double* result);

}  // namespace detail

// The vector CH passes (OP_V1, OP_V2, OP_V1A), instantiated in their own translation units
// (kernels_vch_f32.cu, kernels_vch_f64.cu) so that they compile in parallel with the rest.
template <typename T>
cudaError_t sweep_vch(int axis, const LineParams<T>& lp, int kind, const OpArgs<T>& a, int nx, int ny,
                      ColScratch<T>* cs, unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof);

// The 2D iteration passes 1-4, each instantiated in a translation unit of its own
// (kernels_p1.cu .. kernels_p4.cu) so that they compile in parallel with the rest.
#define MOLT_DECLARE_PASS(fn)                                                                                   \
    template <typename T>                                                                                     \
    cudaError_t fn(int axis, const LineParams<T>& lp, int kind, const OpArgs<T>& a, int nx, int ny,            \
                   ColScratch<T>* cs, unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof);
MOLT_DECLARE_PASS(sweep_p1)
MOLT_DECLARE_PASS(sweep_p2)
MOLT_DECLARE_PASS(sweep_p3)
MOLT_DECLARE_PASS(sweep_p4)
MOLT_DECLARE_PASS(sweep_v1)
MOLT_DECLARE_PASS(sweep_v2)
MOLT_DECLARE_PASS(sweep_c3)   // the 3D x-line combination (kernels_c3.cu)
#undef MOLT_DECLARE_PASS

template <typename T>
cudaError_t sweep(int axis, const LineParams<T>& lp, int kind, const OpArgs<T>& a, int nx, int ny, ColScratch<T>* cs,
                  unsigned long long* red, cudaStream_t st, long long* launches, Prof* prof) {
    using namespace detail;
    switch (kind) {
        case OP_COPY: return dispatch<T, OpCopy<T>>(axis, lp, a, nx, ny, cs, red, st, launches, prof, kind);
        case OP_P1: return sweep_p1<T>(axis, lp, kind, a, nx, ny, cs, red, st, launches, prof);
        case OP_P2: return sweep_p2<T>(axis, lp, kind, a, nx, ny, cs, red, st, launches, prof);
        case OP_P3: return sweep_p3<T>(axis, lp, kind, a, nx, ny, cs, red, st, launches, prof);
        case OP_P4: return sweep_p4<T>(axis, lp, kind, a, nx, ny, cs, red, st, launches, prof);
        case OP_1A: return dispatch<T, Op1a<T>>(axis, lp, a, nx, ny, cs, red, st, launches, prof, kind);
        case OP_1B: return dispatch<T, Op1b<T>>(axis, lp, a, nx, ny, cs, red, st, launches, prof, kind);
        case OP_V1:
        case OP_V2:
        case OP_V1A: return sweep_vch<T>(axis, lp, kind, a, nx, ny, cs, red, st, launches, prof);
        case OP_C3: return sweep_c3<T>(axis, lp, kind, a, nx, ny, cs, red, st, launches, prof);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
int max_row_length(int nf) {
    // one line per block: nf * (n + n/32 + 1) * sizeof(T) <= 227 KB; TL <= 1024 with K = 8
    // (two fields) or K = 16 (one field)
    long long n = nf == 1 ? 16384 : 8192;
    while (n > 8 && static_cast<long long>(nf) * (n + (n >> 5) + 1) * static_cast<long long>(sizeof(T)) >
                        detail::kRowMaxSmem)
        n -= 64;
    return static_cast<int>(n);
}

template <typename T>
cudaError_t lincomb(T* out, long long n, const T* x0, double c0, const T* x1, double c1, const T* x2, double c2,
                    const T* x3, double c3, double c4, cudaStream_t st, long long* launches) {
    if (launches) *launches += 1;
    if constexpr (std::is_same<T, float>::value) {
        auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
        if (n % 4 == 0 && al(out) && al(x0) && al(x1) && al(x2) && al(x3)) {
            long long blocks = (n / 4 + 255) / 256;
            if (blocks > 152 * 8) blocks = 152 * 8;
            if (blocks < 1) blocks = 1;
            detail::lincomb4_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(
                out, n / 4, x0, static_cast<float>(c0), x1, static_cast<float>(c1), x2, static_cast<float>(c2), x3,
                static_cast<float>(c3), static_cast<float>(c4));
            return cudaGetLastError();
        }
    }
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    detail::lincomb_kernel<T><<<static_cast<int>(blocks), 256, 0, st>>>(
        out, n, x0, static_cast<T>(c0), x1, static_cast<T>(c1), x2, static_cast<T>(c2), x3, static_cast<T>(c3),
        static_cast<T>(c4));
    return cudaGetLastError();
}

namespace detail {
template <typename T>
__global__ void fill_pattern_kernel(T* p, long long n, unsigned seed, double lo, double hi) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        unsigned long long z = static_cast<unsigned long long>(i) + 0x9E3779B97F4A7C15ull * (seed + 1ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        p[i] = static_cast<T>(lo + (hi - lo) * static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0));
    }
}

// One row j per blockIdx.y; the row weights a[k][j] are loaded once per thread.
template <typename T>
__global__ void add_separable_kernel(T* y, int nx, const Separable s) {
    const int j = blockIdx.y;
    double aj[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) aj[k] = k < s.terms ? s.a[k][j] : 0.0;
    T* row = y + static_cast<size_t>(j) * nx;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
        double acc = static_cast<double>(row[i]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < s.terms) acc = fma(aj[k], s.b[k][i], acc);
        row[i] = static_cast<T>(acc);
    }
}

template <typename T>
__global__ void cubic_kernel(T* out, long long n, const T* x, T a2, T a1) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const T v = x[i];
        out[i] = v * fma(v, v + a2, a1);
    }
}
}  // namespace detail

namespace detail {
// Sixth-order model: f = v^3 - 3v^2 + 2v and p = -eps2 f'(v) lap + f f'(v) - eta_eps2 f, with
// f'(v) = 3v^2 - 6v + 2 (the pointwise part of the lagged term).
template <typename T>
__global__ void fch_pointwise_kernel(long long n, const T* __restrict__ v, const T* __restrict__ lap, T eps2,
                                     T eta_eps2, T* __restrict__ f_out, T* __restrict__ p_out) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const T x = v[i];
        const T f = x * fma(x, x - T(3), T(2));
        const T fp = fma(x, fma(T(3), x, T(-6)), T(2));
        f_out[i] = f;
        p_out[i] = fma(f, fp, -fma(eps2 * fp, lap[i], eta_eps2 * f));
    }
}
}  // namespace detail

template <typename T>
cudaError_t fch_pointwise(long long n, const T* v, const T* lap, double eps2, double eta_eps2, T* f_out, T* p_out,
                          cudaStream_t st, long long* launches) {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    detail::fch_pointwise_kernel<T><<<static_cast<int>(blocks), 256, 0, st>>>(
        n, v, lap, static_cast<T>(eps2), static_cast<T>(eta_eps2), f_out, p_out);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

namespace detail {
template <typename T>
__global__ void set_walls_kernel(T* w, int nx, int ny, T value) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (ny == 1) {
        if (t == 0) w[0] = value;
        if (t == 1) w[nx - 1] = value;
        return;
    }
    if (t < nx) {
        w[t] = value;                                          // row 0
        w[static_cast<size_t>(ny - 1) * nx + t] = value;       // row ny - 1
    } else if (t < nx + ny) {
        const size_t j = static_cast<size_t>(t - nx);
        w[j * nx] = value;                                     // column 0
        w[j * nx + nx - 1] = value;                            // column nx - 1
    }
}
}  // namespace detail

template <typename T>
cudaError_t set_walls(T* w, int nx, int ny, double value, cudaStream_t st, long long* launches) {
    const int total = ny == 1 ? 2 : nx + ny;
    detail::set_walls_kernel<T><<<(total + 255) / 256, 256, 0, st>>>(w, nx, ny, static_cast<T>(value));
    if (launches) *launches += 1;
    return cudaGetLastError();
}

template <typename T>
cudaError_t fill_pattern(T* p, long long n, unsigned seed, double lo, double hi, cudaStream_t st) {
    detail::fill_pattern_kernel<T><<<152 * 4, 256, 0, st>>>(p, n, seed, lo, hi);
    return cudaGetLastError();
}

template <typename T>
cudaError_t add_separable(T* y, int nx, int ny, const Separable& s, cudaStream_t st, long long* launches) {
    if (s.terms < 1 || s.terms > 4 || ny > 65535) return cudaErrorInvalidValue;
    const int bx = nx >= 2048 ? 8 : (nx + 255) / 256;
    detail::add_separable_kernel<T><<<dim3(bx, ny), 256, 0, st>>>(y, nx, s);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

template <typename T>
cudaError_t cubic(T* out, long long n, const T* x, double a2, double a1, cudaStream_t st, long long* launches) {
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    detail::cubic_kernel<T><<<static_cast<int>(blocks), 256, 0, st>>>(out, n, x, static_cast<T>(a2),
                                                                      static_cast<T>(a1));
    if (launches) *launches += 1;
    return cudaGetLastError();
}

template <typename T>
cudaError_t energy_mass(const T* u, int nx, int ny, int bc, double hx, double hy, double eps, int which,
                        double* partials, double* result, cudaStream_t st, long long* launches) {
    detail::energy_mass_kernel<T><<<detail::kRedBlocks, detail::kRedThreads, 0, st>>>(u, nx, ny, bc, hx, hy, eps,
                                                                                      which, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    detail::sum_partials_kernel<<<1, detail::kRedThreads, 0, st>>>(partials, detail::kRedBlocks, result);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

}  // namespace molt

namespace molt {
namespace detail {

// max |a - b| over n values.  Each |a_i - b_i| and the running max are formed in the field
// precision: rounding is monotone, so the FP32 result is the FP32 rounding of the exact maximum
// (for the nearby iterates a residual compares, the difference is exact), and the loop stays a
// memory stream instead of an FP64 one.  The thread's max is widened to FP64 for the combine; the
// non-negative FP64 bit patterns order like the values, so blocks combine by an integer atomicMax
// on *out (zeroed by the caller).
template <typename T>
__global__ void max_abs_diff_kernel(const T* __restrict__ a, const T* __restrict__ b, long long n,
                                    unsigned long long* out) {
    T mt = T(0);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        mt = fmax(mt, fabs(a[i] - b[i]));
    double m = static_cast<double>(mt);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    __shared__ double s[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s[warp] = m;
    __syncthreads();
    if (warp == 0) {
        m = lane < static_cast<int>(blockDim.x >> 5) ? s[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
        if (lane == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(m)));
    }
}

}  // namespace detail

template <typename T>
cudaError_t max_abs_diff(const T* a, const T* b, long long n, unsigned long long* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    detail::max_abs_diff_kernel<T><<<detail::kRedBlocks, 256, 0, st>>>(a, b, n, out);
    return cudaGetLastError();
}

}  // namespace molt

#define MOLT_INSTANTIATE(T)                                                                                   \
    template cudaError_t molt::sweep<T>(int, const molt::LineParams<T>&, int, const molt::OpArgs<T>&, int, int, \
                                        molt::ColScratch<T>*, unsigned long long*, cudaStream_t, long long*,    \
                                        molt::Prof*);                                                           \
    template int molt::max_row_length<T>(int);                                                                \
    template cudaError_t molt::lincomb<T>(T*, long long, const T*, double, const T*, double, const T*, double,  \
                                          const T*, double, double, cudaStream_t, long long*);                  \
    template cudaError_t molt::energy_mass<T>(const T*, int, int, int, double, double, double, int, double*,    \
                                              double*, cudaStream_t, long long*);                               \
    template cudaError_t molt::cubic<T>(T*, long long, const T*, double, double, cudaStream_t, long long*);    \
    template cudaError_t molt::add_separable<T>(T*, int, int, const molt::Separable&, cudaStream_t, long long*); \
    template cudaError_t molt::fill_pattern<T>(T*, long long, unsigned, double, double, cudaStream_t);         \
    template cudaError_t molt::set_walls<T>(T*, int, int, double, cudaStream_t, long long*);                   \
    template cudaError_t molt::max_abs_diff<T>(const T*, const T*, long long, unsigned long long*, cudaStream_t); \
    template cudaError_t molt::fch_pointwise<T>(long long, const T*, const T*, double, double, T*, T*, cudaStream_t, \
                                                long long*);
