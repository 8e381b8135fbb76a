// Batched 2D Cahn-Hilliard steps in FP32: many independent instances, each with its own grid
// size, eps and time step, advanced together.
//
// Every pass of the stage solve (the rhs inverse Y = M_o^{-1} M_i^{-1} r and the four passes of
// each fixed-point iteration, Sec. 5) is ONE launch over all instances, driven by work lists
// built when the batch is created: a row item is a block of lines of one instance, a column
// item one 128-row tile of a 32-column strip, a carry item 128 columns of one instance.  Each
// block copies its instance's line parameters (Sec. 3.2 weights, boundary coefficients) into
// shared memory and runs the same block bodies as the single-instance general kernels.  Each
// instance has its own stage coefficients, residual slots and stopping state (the rule of the
// single-instance loop); instances that have stopped skip the remaining iterations.  The stage
// of one step (field loads, rhs inverse, the fixed-point loop as a conditional WHILE node, the
// field store) is one CUDA graph.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/molt.h"
#include "molt_internal.h"
#include "sweep_kernels.cuh"

namespace molt {
namespace batch {

constexpr int kRowThreads = 128;   // block of the row passes (lines of at most 1024 nodes)
constexpr int kRowK = 8;           // positions per thread in a row
constexpr int kColKY = 16, kColWY = 8, kColR = kColKY * kColWY;
constexpr int kCarryThreads = 128;
enum Slot { LIX = 0, LOX = 1, LIY = 2, LOY = 3 };   // line parameters: axis x / y, inner / outer c

struct Inst {
    int nx, ny, tiles;
    int aoff;         // offset of the instance's rows in the packed Dirichlet offset row weights
    long long off;    // element offset of the instance in a packed field
    long long soff;   // element offset of the instance in each column-scan scratch array
    int boff;         // offset of the instance's columns in the packed Dirichlet offset profiles
    int pad;
};
struct RowRef {
    int inst, row;
};
struct Stage {
    float g2, g1, beta, pad;   // lagged term G(w) = w (w (w + g2) + g1), beta = tau / c_in
};
struct RowItem {
    int inst, line0, lpb, tl_log2, pitch, pad;
};
struct ColItem {
    int inst, strip, tile, pad;
};
struct CarryItem {
    int inst, idx0;
};

// Instance placement of the fused ops: field pointers + the instance offset, stage coefficients.
__device__ __forceinline__ void place(OpCopy<float>& o, long long off) {
    o.in += off;
    o.out += off;
}
__device__ __forceinline__ void place(OpP1<float>& o, long long off) {
    o.w += off;
    o.t_out += off;
    o.s_out += off;
}
__device__ __forceinline__ void place(OpP2<float>& o, long long off) {
    o.w += off;
    o.t_in += off;
    o.s_in += off;
    o.p_out += off;
    o.u_out += off;
}
__device__ __forceinline__ void place(OpP3<float>& o, long long off) {
    o.p_in += off;
    o.u_in += off;
    o.q1_out += off;
    o.q2_out += off;
}
__device__ __forceinline__ void place(OpP4<float>& o, long long off) {
    o.q1_in += off;
    o.q2_in += off;
    o.u_in += off;
    o.y_in += off;
    o.w += off;
}
__device__ __forceinline__ void coeffs(OpCopy<float>&, const Stage&) {}
__device__ __forceinline__ void coeffs(OpP1<float>& o, const Stage& s) {
    o.g2 = s.g2;
    o.g1 = s.g1;
}
__device__ __forceinline__ void coeffs(OpP2<float>& o, const Stage& s) {
    o.g2 = s.g2;
    o.g1 = s.g1;
    o.beta = s.beta;
}
__device__ __forceinline__ void coeffs(OpP3<float>&, const Stage&) {}
__device__ __forceinline__ void coeffs(OpP4<float>&, const Stage&) {}

// The block's copy of its instance's line parameters.
__device__ __forceinline__ void load_lp(LineParams<float>& dst, const LineParams<float>* src) {
    static_assert(sizeof(LineParams<float>) % 8 == 0, "line parameters are copied in 8-byte words");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x, nt = blockDim.x * blockDim.y;
    for (int i = tid; i < static_cast<int>(sizeof(LineParams<float>) / 8); i += nt) d[i] = s[i];
    __syncthreads();
}

// Every batched kernel walks its work list from item blockIdx.x in steps of gridDim.x, so one
// launch may run one block per item or a persistent grid that loops over the items (the grid size
// is the batch's schedule, chosen by molt_batch_autotune).  The block barrier at the end of each
// item keeps the next item's shared-memory writes behind this item's reads.

template <int M, class Op, bool kLoop>
__global__ void __launch_bounds__(kRowThreads)
rows_batch_kernel(const RowItem* __restrict__ items, int nitems, const Inst* __restrict__ inst,
                  const LineParams<float>* __restrict__ lps, int slot, const Stage* __restrict__ stages,
                  const int* __restrict__ done, const Op op0, unsigned long long* red) {
    __shared__ LineParams<float> slp;
    extern __shared__ __align__(16) unsigned char sm_rows_batch[];
    auto body = [&](int i) {
        const RowItem it = items[i];
        if (done != nullptr && done[it.inst]) return;
        load_lp(slp, lps + 4 * it.inst + slot);
        const Inst in = inst[it.inst];
        Op op = op0;
        place(op, in.off);
        coeffs(op, stages[it.inst]);
        op.ls = in.nx;
        op.ps = 1;
        rows_body<float, M, kRowK, Op>(slp, op, in.ny, it.tl_log2, it.lpb, it.pitch, it.line0,
                                       reinterpret_cast<float*>(sm_rows_batch), red + 2 * it.inst);
    };
    if constexpr (!kLoop) {
        body(blockIdx.x);
    } else {
        for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
            body(i);
            __syncthreads();
        }
    }
}

template <int M, class Op, bool kLoop>
__global__ void __launch_bounds__(32 * kColWY)
cols_agg_batch_kernel(const ColItem* __restrict__ items, int nitems, const Inst* __restrict__ inst,
                      const LineParams<float>* __restrict__ lps, int slot, const Stage* __restrict__ stages,
                      const int* __restrict__ done, const Op op0, float* aggL, float* aggR) {
    __shared__ LineParams<float> slp;
    auto body = [&](int i) {
        const ColItem it = items[i];
        if (done != nullptr && done[it.inst]) return;
        load_lp(slp, lps + 4 * it.inst + slot);
        const Inst in = inst[it.inst];
        Op op = op0;
        place(op, in.off);
        coeffs(op, stages[it.inst]);
        op.ls = 1;
        op.ps = in.nx;
        cols_agg_body<float, M, kColKY, kColWY, Op>(slp, op, in.nx, aggL + in.soff, aggR + in.soff, in.tiles,
                                                    it.strip, it.tile);
    };
    if constexpr (!kLoop) {
        body(blockIdx.x);
    } else {
        for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
            body(i);
            __syncthreads();
        }
    }
}

template <bool kLoop>
__global__ void __launch_bounds__(kCarryThreads)
carry_batch_kernel(const CarryItem* __restrict__ items, int nitems, const Inst* __restrict__ inst,
                   const LineParams<float>* __restrict__ lps, int slot, const int* __restrict__ done, int nf,
                   const float* aggL, const float* aggR, float* carL, float* carR) {
    __shared__ LineParams<float> slp;
    auto body = [&](int i) {
        const CarryItem it = items[i];
        if (done != nullptr && done[it.inst]) return;
        load_lp(slp, lps + 4 * it.inst + slot);
        const Inst in = inst[it.inst];
        carry_body<float>(slp, in.nx, nf, in.tiles, kColR, aggL + in.soff, aggR + in.soff, carL + in.soff,
                          carR + in.soff, it.idx0 + static_cast<int>(threadIdx.x));
    };
    if constexpr (!kLoop) {
        body(blockIdx.x);
    } else {
        for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
            body(i);
            __syncthreads();
        }
    }
}

template <int M, class Op, bool kLoop>
__global__ void __launch_bounds__(32 * kColWY)
cols_final_batch_kernel(const ColItem* __restrict__ items, int nitems, const Inst* __restrict__ inst,
                        const LineParams<float>* __restrict__ lps, int slot, const Stage* __restrict__ stages,
                        const int* __restrict__ done, const Op op0, const float* carL, const float* carR,
                        unsigned long long* red) {
    __shared__ LineParams<float> slp;
    auto body = [&](int i) {
        const ColItem it = items[i];
        if (done != nullptr && done[it.inst]) return;
        load_lp(slp, lps + 4 * it.inst + slot);
        const Inst in = inst[it.inst];
        Op op = op0;
        place(op, in.off);
        coeffs(op, stages[it.inst]);
        op.ls = 1;
        op.ps = in.nx;
        cols_final_body<float, M, kColKY, kColWY, Op>(slp, op, in.nx, carL + in.soff, carR + in.soff, in.tiles,
                                                      it.strip, it.tile, red + 2 * it.inst);
    };
    if constexpr (!kLoop) {
        body(blockIdx.x);
    } else {
        for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
            body(i);
            __syncthreads();
        }
    }
}

__global__ void loop_init_batch_kernel(LoopState* ls, unsigned long long* red, int* done, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        LoopState s;
        s.k = 0;
        s.stall = 0;
        s.done = 0;
        s.converged = 0;
        s.best = __longlong_as_double(0x7ff0000000000000LL);   // +inf
        s.res = s.best;
        s.tol_used = 0.0;
        ls[i] = s;
        red[2 * i] = 0ull;
        red[2 * i + 1] = 0ull;
        done[i] = 0;
    }
}

// Dirichlet batches: Y += the stage's offset C of each instance (molt::dirichlet_offset), one row
// per work item, the sum formed in FP64 in the order of the single-instance add_separable.
__global__ void add_offset_batch_kernel(float* y, const RowRef* __restrict__ rows, int nrows,
                                        const Inst* __restrict__ inst, const double* __restrict__ alpha,
                                        const double* __restrict__ beta, long long astride, long long bstride) {
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const RowRef it = rows[r];
        const Inst in = inst[it.inst];
        double aj[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) aj[k] = alpha[k * astride + in.aoff + it.row];
        float* row = y + in.off + static_cast<long long>(it.row) * in.nx;
        for (int i = threadIdx.x; i < in.nx; i += blockDim.x) {
            double acc = static_cast<double>(row[i]);
#pragma unroll
            for (int k = 0; k < 4; ++k) acc = fma(aj[k], beta[k * bstride + in.boff + i], acc);
            row[i] = static_cast<float>(acc);
        }
    }
}

// Dirichlet batches: the stored wall value w = v - 1 = -1 on the four walls of instance blockIdx.x.
__global__ void walls_batch_kernel(float* w, const Inst* __restrict__ inst, int count) {
    if (static_cast<int>(blockIdx.x) >= count) return;
    const Inst in = inst[blockIdx.x];
    float* f = w + in.off;
    for (int t = threadIdx.x; t < in.nx + in.ny; t += blockDim.x) {
        if (t < in.nx) {
            f[t] = -1.0f;
            f[static_cast<long long>(in.ny - 1) * in.nx + t] = -1.0f;
        } else {
            const long long j = t - in.nx;
            f[j * in.nx] = -1.0f;
            f[j * in.nx + in.nx - 1] = -1.0f;
        }
    }
}

// One block.  Per instance still iterating: the stopping rule of the single-instance loop
// (tolerance floored at 2 ulp of max|w|, the FP32 stall rule, max_iter); then the loop goes on
// while any instance iterates (the WHILE condition in a graph, *active otherwise).
template <bool kGraph>
__global__ void loop_check_batch_kernel(cudaGraphConditionalHandle h, LoopState* ls, unsigned long long* red,
                                        int* done, int n, double tol, int max_iter, int* active_out) {
    int active = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (!done[i]) {
            const double res = __longlong_as_double(static_cast<long long>(red[2 * i]));
            const double wmax = __longlong_as_double(static_cast<long long>(red[2 * i + 1]));
            LoopState s = ls[i];
            s.k += 1;
            const double ulp = wmax * 5.9604644775390625e-08;   // 2^-24 max|w|
            double tol_used = fmax(tol, 2.0 * ulp);
            bool conv = false, stop = false;
            if (!isfinite(res)) {
                stop = true;
            } else if (res < tol_used) {
                conv = true;
            } else if (res < s.best) {
                s.best = res;
                s.stall = 0;
            } else if (res < 64.0 * ulp && ++s.stall >= 6) {
                conv = true;
                tol_used = res;
            }
            s.res = res;
            s.tol_used = tol_used;
            s.converged = conv ? 1 : 0;
            stop = stop || conv || s.k >= max_iter;
            s.done = stop ? 1 : 0;
            ls[i] = s;
            done[i] = s.done;
        }
        red[2 * i] = 0ull;
        red[2 * i + 1] = 0ull;
        active |= done[i] ? 0 : 1;
    }
    active = __syncthreads_or(active);
    if (threadIdx.x == 0) {
        if constexpr (kGraph) cudaGraphSetConditional(h, active ? 1u : 0u);
        else *active_out = active;
    }
}

}  // namespace batch
}  // namespace molt

// =============================================================================================
// Host side
// =============================================================================================
using molt::LineParams;
using molt::LoopState;
using molt::batch::CarryItem;
using molt::batch::ColItem;
using molt::batch::Inst;
using molt::batch::RowItem;
using molt::batch::RowRef;
using molt::batch::Stage;

struct molt_batch {
    int count = 0, bc = 0, M = 4, max_iter = 0;
    double tol = 0.0;
    int exec_mode = MOLT_EXEC_GRAPH;
    std::vector<molt_instance> desc;
    std::vector<Inst> inst_h;
    long long total = 0, scratch = 0;
    int row_smem = 0, n_row = 0, n_col = 0, n_carry[2] = {0, 0};
    int grid_rows = 0, grid_cols = 0;   // schedule: blocks per row / column launch (0 = one per item)
    // device
    Inst* inst = nullptr;
    LineParams<float>* lps = nullptr;   // [count][4] (slots LIX, LOX, LIY, LOY)
    Stage* stages = nullptr;            // [count]
    int* done = nullptr;                // [count]
    int* active = nullptr;              // [1] (host-driven loop)
    LoopState* ls = nullptr;            // [count]
    unsigned long long* red = nullptr;  // [count][2]
    RowItem* rows = nullptr;
    ColItem* cols = nullptr;
    CarryItem* carry[2] = {nullptr, nullptr};
    float *w = nullptr, *r = nullptr, *Y = nullptr, *wprev = nullptr, *f[6] = {};
    float *aggL = nullptr, *aggR = nullptr, *carL = nullptr, *carR = nullptr;
    // Dirichlet batches store u: per-instance offset profiles of the stage (row weights alpha[4][sum ny],
    // column profiles beta[4][sum nx]), the FP64 profile workspace and the row work list
    double *alpha = nullptr, *beta = nullptr, *dprof = nullptr;
    RowRef* yrows = nullptr;
    int n_yrows = 0;
    long long sum_nx = 0, sum_ny = 0;
    std::vector<void*> allocs;
    // pinned host staging
    LineParams<float>* lps_host = nullptr;
    Stage* stages_host = nullptr;
    LoopState* ls_host = nullptr;
    int* active_host = nullptr;
    std::vector<double> tau_loaded;     // taus whose parameters sit in lps / stages
    std::vector<double> applied[4];     // c of the batched sweeps whose parameters sit in each slot
    int applied_last[2] = {0, 2};       // slot (LIX, LIY) of each axis written last by a batched sweep
    bool have_prev = false;
    std::vector<double> dt_prev;
    struct Graph {
        bool valid = false;
        const float* u = nullptr;
        int variant = -1;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
    };
    static constexpr int kGraphs = 4;
    Graph graphs[kGraphs];
    int next_graph = 0;
    cudaStream_t cap = nullptr;
    long long launches = 0;

    void drop_graphs() {
        for (Graph& g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            g = Graph();
        }
    }
    ~molt_batch() {
        drop_graphs();
        if (cap) cudaStreamDestroy(cap);
        for (void* a : allocs) cudaFree(a);
        if (lps_host) cudaFreeHost(lps_host);
        if (stages_host) cudaFreeHost(stages_host);
        if (ls_host) cudaFreeHost(ls_host);
        if (active_host) cudaFreeHost(active_host);
    }
};

namespace {

using namespace molt::batch;

molt_status batch_fail(molt_status s, const std::string& m) {
    molt::set_abi_error(m.c_str());
    return s;
}

template <typename U>
bool balloc(molt_batch* b, U** p, size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, (n ? n : 1) * sizeof(U)) != cudaSuccess) return false;
    b->allocs.push_back(q);
    *p = static_cast<U*>(q);
    return true;
}

// Grid of a pass over n work items under the batch's schedule (0 = one block per item).
inline int pass_grid(int nitems, int cap) { return cap > 0 && cap < nitems ? cap : (nitems > 0 ? nitems : 1); }

// A persistent grid (cap below the item count) runs the looping kernels; one block per item runs
// the single-item kernels, which keep the smaller register footprint of the block bodies.
inline bool loops(int nitems, int cap) { return cap > 0 && cap < nitems; }

template <int M, class Op>
cudaError_t rows_pass(molt_batch* b, int slot, const Op& op, bool skip, cudaStream_t st) {
    const int grid = pass_grid(b->n_row, b->grid_rows);
    const int* dn = skip ? b->done : nullptr;
    if (loops(b->n_row, b->grid_rows))
        rows_batch_kernel<M, Op, true><<<grid, kRowThreads, b->row_smem, st>>>(b->rows, b->n_row, b->inst, b->lps, slot,
                                                                              b->stages, dn, op, b->red);
    else
        rows_batch_kernel<M, Op, false><<<grid, kRowThreads, b->row_smem, st>>>(b->rows, b->n_row, b->inst, b->lps,
                                                                               slot, b->stages, dn, op, b->red);
    b->launches += 1;
    return cudaGetLastError();
}

template <int M, class Op, bool kLoop>
void cols_launch(molt_batch* b, int slot, const Op& op, const int* dn, cudaStream_t st) {
    constexpr int NF = Op::NF;
    const dim3 blk(32, kColWY);
    const int nc = b->n_carry[NF - 1];
    const int gcol = pass_grid(b->n_col, b->grid_cols), gcar = pass_grid(nc, b->grid_cols);
    cols_agg_batch_kernel<M, Op, kLoop><<<gcol, blk, 0, st>>>(b->cols, b->n_col, b->inst, b->lps, slot, b->stages, dn,
                                                              op, b->aggL, b->aggR);
    if (loops(nc, b->grid_cols))
        carry_batch_kernel<true><<<gcar, kCarryThreads, 0, st>>>(b->carry[NF - 1], nc, b->inst, b->lps, slot, dn, NF,
                                                                 b->aggL, b->aggR, b->carL, b->carR);
    else
        carry_batch_kernel<false><<<gcar, kCarryThreads, 0, st>>>(b->carry[NF - 1], nc, b->inst, b->lps, slot, dn, NF,
                                                                  b->aggL, b->aggR, b->carL, b->carR);
    cols_final_batch_kernel<M, Op, kLoop><<<gcol, blk, 0, st>>>(b->cols, b->n_col, b->inst, b->lps, slot, b->stages,
                                                                dn, op, b->carL, b->carR, b->red);
}

template <int M, class Op>
cudaError_t cols_pass(molt_batch* b, int slot, const Op& op, bool skip, cudaStream_t st) {
    const int* dn = skip ? b->done : nullptr;
    if (loops(b->n_col, b->grid_cols)) cols_launch<M, Op, true>(b, slot, op, dn, st);
    else cols_launch<M, Op, false>(b, slot, op, dn, st);
    b->launches += 3;
    return cudaGetLastError();
}

// Y = M_o^{-1} M_i^{-1} r with M = H_x H_y (columns first, as in the single-instance solver)
template <int M>
cudaError_t rhs_inverse(molt_batch* b, cudaStream_t st) {
    cudaError_t e;
    molt::OpCopy<float> c{};
    c.in = b->r;
    c.out = b->f[0];
    if ((e = cols_pass<M>(b, LIY, c, false, st)) != cudaSuccess) return e;
    c.in = b->f[0];
    c.out = b->f[1];
    if ((e = rows_pass<M>(b, LIX, c, false, st)) != cudaSuccess) return e;
    c.in = b->f[1];
    c.out = b->f[0];
    if ((e = cols_pass<M>(b, LOY, c, false, st)) != cudaSuccess) return e;
    c.in = b->f[0];
    c.out = b->Y;
    return rows_pass<M>(b, LOX, c, false, st);
}

// One fixed-point iteration of every instance still iterating (passes 1-4 of the 2D iteration).
template <int M>
cudaError_t iteration(molt_batch* b, cudaStream_t st) {
    cudaError_t e;
    molt::OpP1<float> a1{};
    a1.w = b->w;
    a1.t_out = b->f[0];
    a1.s_out = b->f[1];
    if ((e = cols_pass<M>(b, LIY, a1, true, st)) != cudaSuccess) return e;
    molt::OpP2<float> a2{};
    a2.w = b->w;
    a2.t_in = b->f[0];
    a2.s_in = b->f[1];
    a2.p_out = b->f[2];
    a2.u_out = b->f[3];
    if ((e = rows_pass<M>(b, LIX, a2, true, st)) != cudaSuccess) return e;
    molt::OpP3<float> a3{};
    a3.p_in = b->f[2];
    a3.u_in = b->f[3];
    a3.q1_out = b->f[4];
    a3.q2_out = b->f[5];
    if ((e = cols_pass<M>(b, LOY, a3, true, st)) != cudaSuccess) return e;
    molt::OpP4<float> a4{};
    a4.q1_in = b->f[4];
    a4.q2_in = b->f[5];
    a4.u_in = b->f[3];
    a4.y_in = b->Y;
    a4.w = b->w;
    cudaError_t e4 = rows_pass<M>(b, LOX, a4, true, st);
    if (e4 != cudaSuccess || b->bc != molt::BC_DIRICHLET) return e4;
    // every Dirichlet line inverse holds v = 0 on the walls: the stored w = -1 is set there, as the
    // single-instance solver does after each iteration
    walls_batch_kernel<<<b->count, 256, 0, st>>>(b->w, b->inst, b->count);
    b->launches += 1;
    return cudaGetLastError();
}

cudaError_t rhs_inverse_any(molt_batch* b, cudaStream_t st) {
    switch (b->M) {
        case 2: return rhs_inverse<2>(b, st);
        case 4: return rhs_inverse<4>(b, st);
        default: return rhs_inverse<6>(b, st);
    }
}
cudaError_t iteration_any(molt_batch* b, cudaStream_t st) {
    switch (b->M) {
        case 2: return iteration<2>(b, st);
        case 4: return iteration<4>(b, st);
        default: return iteration<6>(b, st);
    }
}

// One line inversion H_c of every instance along one axis, with the parameters of c_i held in
// `slot` (LIX or LOX for x, LIY or LOY for y) while it runs.
template <int M>
cudaError_t apply_pass(molt_batch* b, int axis, int slot, const float* in, float* out, cudaStream_t st) {
    molt::OpCopy<float> c{};
    c.in = in;
    c.out = out;
    return axis == 0 ? rows_pass<M>(b, slot, c, false, st) : cols_pass<M>(b, slot, c, false, st);
}

cudaError_t lin(molt_batch* b, float* out, const float* x0, double c0, const float* x1, double c1, double c4,
                cudaStream_t st) {
    return molt::lincomb<float>(out, b->total, x0, c0, x1, c1, nullptr, 0.0, nullptr, 0.0, c4, st, &b->launches);
}

// Step variants: 0 = BE, 1 = BE that also keeps the BDF2 history, 2 = BDF2 with history.
// Stored variable w = u = v - 1 on every grid (as the single-instance solver; Dirichlet stages add
// their offset to Y).
cudaError_t pre_ops(molt_batch* b, const float* u, int variant, cudaStream_t st) {
    cudaError_t e;
    if ((e = lin(b, b->w, u, 1.0, nullptr, 0.0, 0.0, st)) != cudaSuccess) return e;
    if (variant == 2) {
        if ((e = lin(b, b->r, b->w, 4.0 / 3.0, b->wprev, -1.0 / 3.0, 0.0, st)) != cudaSuccess) return e;
    } else {
        if ((e = lin(b, b->r, b->w, 1.0, nullptr, 0.0, 0.0, st)) != cudaSuccess) return e;
    }
    if (variant >= 1 && (e = lin(b, b->wprev, b->w, 1.0, nullptr, 0.0, 0.0, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t post_ops(molt_batch* b, float* u, cudaStream_t st) { return lin(b, u, b->w, 1.0, nullptr, 0.0, 0.0, st); }

// Y of every instance, with the Dirichlet offsets of the loaded stage parameters.
cudaError_t rhs_with_offset(molt_batch* b, cudaStream_t st) {
    cudaError_t e = rhs_inverse_any(b, st);
    if (e != cudaSuccess || b->bc != molt::BC_DIRICHLET) return e;
    add_offset_batch_kernel<<<b->n_yrows < 152 * 8 ? b->n_yrows : 152 * 8, 128, 0, st>>>(
        b->Y, b->yrows, b->n_yrows, b->inst, b->alpha, b->beta, b->sum_ny, b->sum_nx);
    b->launches += 1;
    return cudaGetLastError();
}

cudaError_t loop_init(molt_batch* b, cudaStream_t st) {
    loop_init_batch_kernel<<<(b->count + 255) / 256, 256, 0, st>>>(b->ls, b->red, b->done, b->count);
    b->launches += 1;
    return cudaGetLastError();
}

// Stage parameters of every instance for the given taus (line parameters in the FP64 host
// build of the single-instance solver, cast to FP32), uploaded when they change.
molt_status load_params(molt_batch* b, const std::vector<double>& tau, cudaStream_t st) {
    if (tau == b->tau_loaded) return MOLT_OK;
    const double s = 1.0;   // stored w = v - 1 on every grid
    for (int i = 0; i < b->count; ++i) {
        const molt_instance& d = b->desc[i];
        const molt::StageParams sp = molt::stage_params(tau[i], d.eps);
        const double cs[4] = {sp.c_in, sp.c_out, sp.c_in, sp.c_out};
        for (int slot = 0; slot < 4; ++slot) {
            const bool y = slot >= LIY;
            const int n = y ? d.ny : d.nx;
            const double L = y ? d.Ly : d.Lx;
            molt::LineParams<double> lpd;
            const char* err = nullptr;
            if (!molt::build_line_params(cs[slot], molt::grid_h(n, L, b->bc), n, b->M, b->bc, &lpd, &err))
                return batch_fail(MOLT_ERR_ARG, std::string("instance ") + std::to_string(i) + ": " +
                                                    (err ? err : "bad line parameters"));
            b->lps_host[4 * i + slot] = molt::cast_line_params<float>(lpd);
        }
        Stage st_i;
        st_i.g2 = s == 1.0 ? 0.0f : -3.0f;
        st_i.g1 = s == 1.0 ? static_cast<float>(sp.lam - 3.0) : static_cast<float>(sp.lam);
        st_i.beta = static_cast<float>(sp.beta);
        st_i.pad = 0.0f;
        b->stages_host[i] = st_i;
        if (b->bc == molt::BC_DIRICHLET) {
            // this instance's Y offset (the single-instance profiles), packed by instance
            molt::LineParams<double> lp[4];
            for (int slot = 0; slot < 4; ++slot) {
                const bool y = slot >= LIY;
                const int n = y ? d.ny : d.nx;
                const char* err = nullptr;
                molt::build_line_params(cs[slot], molt::grid_h(n, y ? d.Ly : d.Lx, b->bc), n, b->M, b->bc, &lp[slot],
                                        &err);
            }
            molt::Separable sep;
            cudaError_t e = molt::dirichlet_offset(lp, 2, sp.beta * (sp.lam - 2.0), b->dprof, 1024, &sep, st,
                                                   &b->launches);
            const Inst& in = b->inst_h[i];
            for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
                e = cudaMemcpyAsync(b->alpha + k * b->sum_ny + in.aoff, sep.a[k], sizeof(double) * d.ny,
                                    cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(b->beta + k * b->sum_nx + in.boff, sep.b[k], sizeof(double) * d.nx,
                                        cudaMemcpyDeviceToDevice, st);
            }
            if (e != cudaSuccess)
                return batch_fail(MOLT_ERR_CUDA, std::string("Dirichlet offsets: ") + cudaGetErrorString(e));
        }
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->lps, b->lps_host, sizeof(LineParams<float>) * 4 * b->count, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->stages, b->stages_host, sizeof(Stage) * b->count, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return batch_fail(MOLT_ERR_CUDA, std::string("parameter upload: ") + cudaGetErrorString(e));
    // the pinned staging buffers are rewritten only after this copy has completed
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return batch_fail(MOLT_ERR_CUDA, std::string("parameter upload: ") + cudaGetErrorString(e));
    b->tau_loaded = tau;
    for (std::vector<double>& a : b->applied) a.clear();
    return MOLT_OK;
}

// The step of one variant as a graph: loads and rhs inverse, a conditional WHILE node whose body
// is one iteration plus the per-instance stopping check, the store of u.
molt_batch::Graph* step_graph(molt_batch* b, float* u, int variant) {
    for (molt_batch::Graph& g : b->graphs)
        if (g.valid && g.u == u && g.variant == variant) return &g;
    molt_batch::Graph& g = b->graphs[b->next_graph];
    b->next_graph = (b->next_graph + 1) % molt_batch::kGraphs;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = molt_batch::Graph();
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    const long long launches0 = b->launches;
    cudaGraph_t graph = nullptr, head = nullptr, tail = nullptr;
    bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
    // head: loads, rhs inverse, loop state reset
    if (ok) ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
        const bool launched = pre_ops(b, u, variant, b->cap) == cudaSuccess && rhs_with_offset(b, b->cap) == cudaSuccess &&
                              loop_init(b, b->cap) == cudaSuccess;
        ok = cudaStreamEndCapture(b->cap, &head) == cudaSuccess && launched;
    }
    cudaGraphNode_t n_head = nullptr, n_loop = nullptr, n_tail = nullptr;
    if (ok) ok = cudaGraphAddChildGraphNode(&n_head, graph, nullptr, 0, head) == cudaSuccess;
    // the loop
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams np = {};
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ok = cudaGraphAddNode(&n_loop, graph, &n_head, nullptr, 1, &np) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
             cudaSuccess;
        if (ok) {
            bool launched = iteration_any(b, b->cap) == cudaSuccess;
            if (launched) {
                loop_check_batch_kernel<true><<<1, 1024, 0, b->cap>>>(h, b->ls, b->red, b->done, b->count, b->tol,
                                                                       b->max_iter, nullptr);
                launched = cudaGetLastError() == cudaSuccess;
            }
            cudaGraph_t captured = nullptr;
            ok = cudaStreamEndCapture(b->cap, &captured) == cudaSuccess && launched;
        }
    }
    // tail: store u
    if (ok) ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
        const bool launched = post_ops(b, u, b->cap) == cudaSuccess;
        ok = cudaStreamEndCapture(b->cap, &tail) == cudaSuccess && launched;
    }
    if (ok) ok = cudaGraphAddChildGraphNode(&n_tail, graph, &n_loop, 1, tail) == cudaSuccess;
    cudaGraphExec_t exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (head) cudaGraphDestroy(head);
    if (tail) cudaGraphDestroy(tail);
    b->launches = launches0;
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return nullptr;
    }
    g.valid = true;
    g.u = u;
    g.variant = variant;
    g.graph = graph;
    g.exec = exec;
    return &g;
}

molt_status run_step(molt_batch* b, float* u, int variant, cudaStream_t st) {
    cudaError_t e;
    if (b->exec_mode == MOLT_EXEC_GRAPH) {
        molt_batch::Graph* g = step_graph(b, u, variant);
        if (!g) return batch_fail(MOLT_ERR_CUDA, "building the batch step graph failed");
        if ((e = cudaGraphLaunch(g->exec, st)) != cudaSuccess)
            return batch_fail(MOLT_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    } else {
        if ((e = pre_ops(b, u, variant, st)) != cudaSuccess || (e = rhs_with_offset(b, st)) != cudaSuccess ||
            (e = loop_init(b, st)) != cudaSuccess)
            return batch_fail(MOLT_ERR_CUDA, std::string("stage set-up: ") + cudaGetErrorString(e));
        for (int k = 1; k <= b->max_iter; ++k) {
            if ((e = iteration_any(b, st)) != cudaSuccess)
                return batch_fail(MOLT_ERR_CUDA, std::string("iteration: ") + cudaGetErrorString(e));
            loop_check_batch_kernel<false><<<1, 1024, 0, st>>>(cudaGraphConditionalHandle{}, b->ls, b->red, b->done,
                                                               b->count, b->tol, b->max_iter, b->active);
            if ((e = cudaGetLastError()) != cudaSuccess ||
                (e = cudaMemcpyAsync(b->active_host, b->active, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return batch_fail(MOLT_ERR_CUDA, std::string("loop check: ") + cudaGetErrorString(e));
            b->launches += 1;
            if (!*b->active_host) break;
        }
        if ((e = post_ops(b, u, st)) != cudaSuccess)
            return batch_fail(MOLT_ERR_CUDA, std::string("store: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(b->ls_host, b->ls, sizeof(LoopState) * b->count, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return batch_fail(MOLT_ERR_CUDA, std::string("loop state copy: ") + cudaGetErrorString(e));
    return MOLT_OK;
}

}  // namespace

extern "C" {

molt_status molt_batch_create(molt_batch** out, int count, const molt_instance* instances, molt_bc bc,
                              int quad_order, double tol, int max_iter) {
    if (!out) return batch_fail(MOLT_ERR_ARG, "null output handle");
    *out = nullptr;
    if (count < 1 || !instances) return batch_fail(MOLT_ERR_ARG, "a batch needs at least one instance");
    if (bc < MOLT_BC_PERIODIC || bc > MOLT_BC_DIRICHLET) return batch_fail(MOLT_ERR_ARG, "unknown boundary condition");
    if (quad_order != 2 && quad_order != 4 && quad_order != 6) return batch_fail(MOLT_ERR_ARG, "M must be 2, 4 or 6");
    if (!(tol > 0.0) || max_iter < 1) return batch_fail(MOLT_ERR_ARG, "tol must be > 0 and max_iter >= 1");
    for (int i = 0; i < count; ++i) {
        const molt_instance& d = instances[i];
        if (d.nx < quad_order + 2 || d.ny < quad_order + 2 || d.nx > 1024 || d.ny > 1024)
            return batch_fail(MOLT_ERR_ARG, "instance " + std::to_string(i) + ": nx, ny must lie in [M + 2, 1024]");
        if (!(d.Lx > 0.0) || !(d.Ly > 0.0) || !(d.eps > 0.0) || !std::isfinite(d.Lx) || !std::isfinite(d.Ly) ||
            !std::isfinite(d.eps))
            return batch_fail(MOLT_ERR_ARG, "instance " + std::to_string(i) + ": Lx, Ly, eps must be finite and > 0");
    }
    molt_batch* b = new (std::nothrow) molt_batch();
    if (!b) return batch_fail(MOLT_ERR_OOM, "host allocation failed");
    b->count = count;
    b->bc = bc;
    b->M = quad_order;
    b->tol = tol;
    b->max_iter = max_iter;
    b->desc.assign(instances, instances + count);
    std::vector<RowItem> rows;
    std::vector<ColItem> cols;
    std::vector<CarryItem> carry[2];
    std::vector<RowRef> yrows;
    long long off = 0, soff = 0;
    for (int i = 0; i < count; ++i) {
        const molt_instance& d = instances[i];
        Inst in{};
        in.nx = d.nx;
        in.ny = d.ny;
        in.tiles = (d.ny + kColR - 1) / kColR;
        in.off = off;
        in.soff = soff;
        in.aoff = static_cast<int>(b->sum_ny);
        in.boff = static_cast<int>(b->sum_nx);
        off += static_cast<long long>(d.nx) * d.ny;
        soff += 2LL * in.tiles * d.nx;
        b->sum_ny += d.ny;
        b->sum_nx += d.nx;
        b->inst_h.push_back(in);
        if (bc == MOLT_BC_DIRICHLET)
            for (int j = 0; j < d.ny; ++j) yrows.push_back({i, j});
        // rows: the general row kernel's team (K = 8 positions per thread), lpb lines per block
        int tl_log2 = 0;
        while ((1 << tl_log2) < (d.nx + kRowK - 1) / kRowK) ++tl_log2;
        const int TL = 1 << tl_log2;
        const int lpb = kRowThreads / TL;
        const int pitch = d.nx + (d.nx >> 5) + 1;
        b->row_smem = std::max(b->row_smem, static_cast<int>(lpb * 2 * pitch * sizeof(float)));
        for (int l0 = 0; l0 < d.ny; l0 += lpb) rows.push_back({i, l0, lpb, tl_log2, pitch, 0});
        for (int t = 0; t < in.tiles; ++t)
            for (int s = 0; s < (d.nx + 31) / 32; ++s) cols.push_back({i, s, t, 0});
        for (int nf = 1; nf <= 2; ++nf)
            for (int j = 0; j < d.nx * nf; j += kCarryThreads) carry[nf - 1].push_back({i, j});
    }
    b->total = off;
    b->scratch = soff;
    b->n_row = static_cast<int>(rows.size());
    b->n_col = static_cast<int>(cols.size());
    b->n_carry[0] = static_cast<int>(carry[0].size());
    b->n_carry[1] = static_cast<int>(carry[1].size());
    const size_t nt = static_cast<size_t>(b->total), ns = static_cast<size_t>(b->scratch);
    bool ok = balloc(b, &b->inst, count) && balloc(b, &b->lps, 4 * static_cast<size_t>(count)) &&
              balloc(b, &b->stages, count) && balloc(b, &b->done, count) && balloc(b, &b->active, 1) &&
              balloc(b, &b->ls, count) && balloc(b, &b->red, 2 * static_cast<size_t>(count)) &&
              balloc(b, &b->rows, rows.size()) && balloc(b, &b->cols, cols.size()) &&
              balloc(b, &b->carry[0], carry[0].size()) && balloc(b, &b->carry[1], carry[1].size()) &&
              balloc(b, &b->w, nt) && balloc(b, &b->r, nt) && balloc(b, &b->Y, nt) && balloc(b, &b->wprev, nt) &&
              balloc(b, &b->aggL, ns) && balloc(b, &b->aggR, ns) && balloc(b, &b->carL, ns) &&
              balloc(b, &b->carR, ns);
    for (int k = 0; ok && k < 6; ++k) ok = balloc(b, &b->f[k], nt);
    if (ok && bc == MOLT_BC_DIRICHLET) {
        b->n_yrows = static_cast<int>(yrows.size());
        ok = balloc(b, &b->alpha, 4 * static_cast<size_t>(b->sum_ny)) &&
             balloc(b, &b->beta, 4 * static_cast<size_t>(b->sum_nx)) &&
             balloc(b, &b->dprof, static_cast<size_t>(molt::kOffsetProfiles) * 1024) &&
             balloc(b, &b->yrows, yrows.size()) &&
             cudaMemcpy(b->yrows, yrows.data(), sizeof(RowRef) * yrows.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
        delete b;
        return batch_fail(MOLT_ERR_OOM, "device workspace allocation failed");
    }
    if (cudaMallocHost(&b->lps_host, sizeof(LineParams<float>) * 4 * count) != cudaSuccess ||
        cudaMallocHost(&b->stages_host, sizeof(Stage) * count) != cudaSuccess ||
        cudaMallocHost(&b->ls_host, sizeof(LoopState) * count) != cudaSuccess ||
        cudaMallocHost(&b->active_host, sizeof(int)) != cudaSuccess) {
        delete b;
        return batch_fail(MOLT_ERR_OOM, "pinned host allocation failed");
    }
    if (cudaMemcpy(b->inst, b->inst_h.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->rows, rows.data(), sizeof(RowItem) * rows.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->cols, cols.data(), sizeof(ColItem) * cols.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->carry[0], carry[0].data(), sizeof(CarryItem) * carry[0].size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->carry[1], carry[1].data(), sizeof(CarryItem) * carry[1].size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        delete b;
        return batch_fail(MOLT_ERR_CUDA, "work list upload failed");
    }
    *out = b;
    return MOLT_OK;
}

molt_status molt_batch_destroy(molt_batch* b) {
    delete b;
    return MOLT_OK;
}

long long molt_batch_points(const molt_batch* b) { return b ? b->total : 0; }

molt_status molt_batch_offsets(const molt_batch* b, long long* offsets) {
    if (!b || !offsets) return batch_fail(MOLT_ERR_ARG, "null batch or output");
    for (int i = 0; i < b->count; ++i) offsets[i] = b->inst_h[i].off;
    return MOLT_OK;
}

molt_status molt_batch_set_execution(molt_batch* b, molt_execution mode) {
    if (!b) return batch_fail(MOLT_ERR_ARG, "null batch");
    if (mode != MOLT_EXEC_HOST_LOOP && mode != MOLT_EXEC_GRAPH) return batch_fail(MOLT_ERR_ARG, "unknown mode");
    b->exec_mode = mode;
    return MOLT_OK;
}

molt_status molt_batch_step(molt_batch* b, float* u, const double* dt, molt_scheme scheme, void* stream, int* iters,
                            double* residual, int* status) {
    if (!b || !u || !dt) return batch_fail(MOLT_ERR_ARG, "null batch, field or dt");
    if (scheme != MOLT_BE && scheme != MOLT_BDF2)
        return batch_fail(MOLT_ERR_UNSUPPORTED, "batched steps support BE and BDF2");
    std::vector<double> dtv(dt, dt + b->count);
    for (int i = 0; i < b->count; ++i)
        if (!(dtv[i] > 0.0) || !std::isfinite(dtv[i]))
            return batch_fail(MOLT_ERR_ARG, "instance " + std::to_string(i) + ": dt must be finite and > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool bdf = scheme == MOLT_BDF2 && b->have_prev && dtv == b->dt_prev;
    const int variant = scheme == MOLT_BE ? 0 : (bdf ? 2 : 1);
    std::vector<double> tau(b->count);
    for (int i = 0; i < b->count; ++i) tau[i] = bdf ? 2.0 * dtv[i] / 3.0 : dtv[i];
    molt_status s = load_params(b, tau, st);
    if (s != MOLT_OK) return s;
    if ((s = run_step(b, u, variant, st)) != MOLT_OK) return s;
    b->have_prev = scheme == MOLT_BDF2;
    b->dt_prev = dtv;
    molt_status worst = MOLT_OK;
    for (int i = 0; i < b->count; ++i) {
        const LoopState& L = b->ls_host[i];
        const molt_status si = L.converged ? MOLT_OK : MOLT_ERR_NOT_CONVERGED;
        if (iters) iters[i] = L.k;
        if (residual) residual[i] = L.res;
        if (status) status[i] = si;
        if (si != MOLT_OK) worst = si;
    }
    if (worst != MOLT_OK) molt::set_abi_error("an instance reached max_iter before the fixed-point tolerance");
    return worst;
}

molt_status molt_batch_helmholtz_apply(molt_batch* b, int axis, const double* c, const float* in, float* out,
                                       void* stream) {
    if (!b || !c || !in || !out) return batch_fail(MOLT_ERR_ARG, "null batch, c or field");
    if (axis != 0 && axis != 1) return batch_fail(MOLT_ERR_ARG, "axis must be 0 (x) or 1 (y)");
    if (in == out) return batch_fail(MOLT_ERR_ARG, "in and out must not alias");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // two parameter slots per axis: a caller alternating between two values of c (the inner and
    // outer inversions of a stage) uploads each once
    const int pair[2] = {axis == 0 ? LIX : LIY, axis == 0 ? LOX : LOY};
    std::vector<double> cv(c, c + b->count);
    int slot = -1;
    for (int s : pair)
        if (cv == b->applied[s]) slot = s;
    cudaError_t e = cudaSuccess;
    if (slot < 0) {
        slot = b->applied_last[axis] == pair[0] ? pair[1] : pair[0];
        for (int i = 0; i < b->count; ++i) {
            const molt_instance& d = b->desc[i];
            if (!(cv[i] > 0.0) || !std::isfinite(cv[i]))
                return batch_fail(MOLT_ERR_ARG, "instance " + std::to_string(i) + ": c must be finite and > 0");
            const int n = axis == 0 ? d.nx : d.ny;
            molt::LineParams<double> lpd;
            const char* err = nullptr;
            if (!molt::build_line_params(cv[i], molt::grid_h(n, axis == 0 ? d.Lx : d.Ly, b->bc), n, b->M, b->bc,
                                         &lpd, &err))
                return batch_fail(MOLT_ERR_ARG, std::string("instance ") + std::to_string(i) + ": " +
                                                    (err ? err : "bad line parameters"));
            b->lps_host[4 * i + slot] = molt::cast_line_params<float>(lpd);
        }
        b->tau_loaded.clear();   // the slot no longer holds a stage's parameters
        // the whole table (the other slots are unchanged); the pinned staging buffer is free again
        // once the copy has completed
        e = cudaMemcpyAsync(b->lps, b->lps_host, sizeof(LineParams<float>) * 4 * b->count, cudaMemcpyHostToDevice,
                            st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        b->applied[slot] = e == cudaSuccess ? cv : std::vector<double>();
        b->applied_last[axis] = slot;
    }
    if (e == cudaSuccess) {
        switch (b->M) {
            case 2: e = apply_pass<2>(b, axis, slot, in, out, st); break;
            case 4: e = apply_pass<4>(b, axis, slot, in, out, st); break;
            default: e = apply_pass<6>(b, axis, slot, in, out, st); break;
        }
    }
    if (e != cudaSuccess) return batch_fail(MOLT_ERR_CUDA, std::string("batched sweep: ") + cudaGetErrorString(e));
    return MOLT_OK;
}

molt_status molt_batch_set_schedule(molt_batch* b, int grid_rows, int grid_cols) {
    if (!b || grid_rows < 0 || grid_cols < 0) return batch_fail(MOLT_ERR_ARG, "null batch or negative grid");
    b->grid_rows = grid_rows;
    b->grid_cols = grid_cols;
    b->drop_graphs();
    return MOLT_OK;
}

molt_status molt_batch_autotune(molt_batch* b, const double* dt, void* stream, double* ms_table, int* grid_rows,
                                int* grid_cols) {
    if (!b || !dt) return batch_fail(MOLT_ERR_ARG, "null batch or dt");
    std::vector<double> tau(dt, dt + b->count);
    for (int i = 0; i < b->count; ++i)
        if (!(tau[i] > 0.0) || !std::isfinite(tau[i]))
            return batch_fail(MOLT_ERR_ARG, "instance " + std::to_string(i) + ": dt must be finite and > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    molt_status s = load_params(b, tau, st);
    if (s != MOLT_OK) return s;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // candidate schedules: one block per work item, or persistent grids of 2, 4, 8 blocks per SM
    const int caps[4] = {0, 2 * sms, 4 * sms, 8 * sms};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = INFINITY;
    int best_r = 0, best_c = 0;
    // time one fixed-point iteration of every instance under each pair of schedules, from the same
    // finite fields each time
    for (int ir = 0; ir < 4 && e == cudaSuccess; ++ir) {
        for (int ic = 0; ic < 4 && e == cudaSuccess; ++ic) {
            b->grid_rows = caps[ir];
            b->grid_cols = caps[ic];
            float ms = 0.0f;
            if ((e = lin(b, b->w, nullptr, 0.0, nullptr, 0.0, 0.05, st)) != cudaSuccess ||
                (e = lin(b, b->Y, nullptr, 0.0, nullptr, 0.0, 0.05, st)) != cudaSuccess || loop_init(b, st) != cudaSuccess)
                break;
            for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = lin(b, b->f[k], nullptr, 0.0, nullptr, 0.0, 0.01 * k, st);
            if (e != cudaSuccess || (e = iteration_any(b, st)) != cudaSuccess) break;   // warm-up
            if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = iteration_any(b, st);
            if (e != cudaSuccess || (e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
                break;
            const double per = ms / 3.0;
            if (ms_table) ms_table[4 * ir + ic] = per;
            if (per < best) {
                best = per;
                best_r = caps[ir];
                best_c = caps[ic];
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->grid_rows = best_r;
    b->grid_cols = best_c;
    b->drop_graphs();          // graphs captured the previous schedule
    b->have_prev = false;      // the work fields were overwritten
    if (e != cudaSuccess) return batch_fail(MOLT_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    if (grid_rows) *grid_rows = best_r;
    if (grid_cols) *grid_cols = best_c;
    return MOLT_OK;
}

}  // extern "C"
